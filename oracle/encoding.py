"""Multiresolution hash encoding with trilinear interpolation (oracle).

Test infrastructure: only the tests, the smoke check and the benchmark's CPU legs
use it.

The paper replaces frequency encoding with hash encoding (Sec. 1), citing the
multiresolution hash grid of Mueller et al. (Instant-NGP) and NAF, and stresses
that each step touches only the sparse subset of table entries that the sampled
points fall on (abstract, Sec. 1: "local sparse"). It prints no formula, so
this file restates the published Instant-NGP encoding:

* L levels with resolutions in a geometric series from N_min to N_max,
  N_l = floor(N_min * exp(l * (ln N_max - ln N_min) / (L - 1)) + 1e-9)
  (the 1e-9 makes the top level equal N_max where exp() lands a hair below it);
* each level stores T entries of F features; grid vertices are the integer
  points 0..N_l of each axis;
* a level whose (N_l + 1)^3 vertices fit in T is indexed densely,
  idx = cx + cy (N_l + 1) + cz (N_l + 1)^2; otherwise spatially hashed,
  idx = (cx * 1) xor (cy * 2654435761) xor (cz * 805459861) mod T with uint32
  wrap-around (the primes published with Instant-NGP);
* a point's cell corner c = min(floor(x_hat * N_l), N_l - 1) after clamping x_hat
  to [0, 1]; the fractional part w = x_hat * N_l - c; corner bit 0 steps x,
  bit 1 steps y, bit 2 steps z, with weight prod(bit ? w : 1 - w);
* the level feature is the weighted sum of its 8 corner entries, and the
  encoding concatenates levels level-major: h[l * F + f].

Positions, scaled coordinates, cells and fractions are float32 (mirrored with
the GPU bit for bit); weights and features are float64.
"""
from __future__ import annotations

import math

import numpy as np

PRIMES = (np.uint32(1), np.uint32(2654435761), np.uint32(805459861))


def level_resolutions(L, base_res, max_res):
    """Per-level grid resolutions N_l (Python ints)."""
    if L == 1:
        return [int(base_res)]
    step = (math.log(max_res) - math.log(base_res)) / (L - 1)
    return [int(math.floor(base_res * math.exp(l * step) + 1e-9)) for l in range(L)]


def is_dense(res, T):
    return (res + 1) ** 3 <= T


def corners(x, resolutions, T):
    """Corner indices (P, L, 8) uint32 and weights (P, L, 8) float64 for points x (P, 3) f32.

    Also returns the float32 fractions (P, L, 3) for bitwise checks.
    """
    x = np.clip(np.asarray(x, dtype=np.float32), np.float32(0.0), np.float32(1.0))
    P, L = x.shape[0], len(resolutions)
    idx = np.zeros((P, L, 8), dtype=np.uint32)
    wts = np.zeros((P, L, 8), dtype=np.float64)
    fr = np.zeros((P, L, 3), dtype=np.float32)
    mask = np.uint32(T - 1)
    for l, n in enumerate(resolutions):
        p = x * np.float32(n)
        c = np.minimum(np.floor(p).astype(np.int64), n - 1)
        w = (p - c.astype(np.float32)).astype(np.float32)
        fr[:, l, :] = w
        w64 = w.astype(np.float64)
        for corner in range(8):
            b = [(corner >> k) & 1 for k in range(3)]
            cc = (c + np.array(b)[None, :]).astype(np.uint32)
            if is_dense(n, T):
                s = np.uint32(n + 1)
                i = cc[:, 0] + cc[:, 1] * s + cc[:, 2] * s * s
            else:
                i = (cc[:, 0] * PRIMES[0]) ^ (cc[:, 1] * PRIMES[1]) ^ (cc[:, 2] * PRIMES[2])
                i = i & mask
            idx[:, l, corner] = i
            wk = np.ones(P)
            for k in range(3):
                wk = wk * (w64[:, k] if b[k] else (1.0 - w64[:, k]))
            wts[:, l, corner] = wk
    return idx, wts, fr


def encode(x, tables, resolutions, T):
    """Trilinear hash features h (P, L*F) for points x (P, 3); tables (L, T, F) float64."""
    idx, w, _ = corners(x, resolutions, T)
    L, _, F = tables.shape
    h = np.zeros((x.shape[0], L * F))
    for l in range(L):
        g = tables[l][idx[:, l, :]]                  # (P, 8, F)
        h[:, l * F:(l + 1) * F] = np.einsum("pc,pcf->pf", w[:, l, :], g)
    return h


def encode_backward(x, dh, resolutions, T, F):
    """Scatter-add of dL/dh into the tables: dT[l, idx_c, f] += w_c * dh[l*F + f].

    Collisions (two corners or points on one entry) add up, as in the chain rule.
    """
    idx, w, _ = corners(x, resolutions, T)
    L = len(resolutions)
    dT = np.zeros((L, T, F))
    for l in range(L):
        flat = idx[:, l, :].ravel().astype(np.int64)
        for f in range(F):
            contrib = (w[:, l, :] * dh[:, l * F + f][:, None]).ravel()
            dT[l, :, f] = np.bincount(flat, weights=contrib, minlength=T)
    return dT
