"""Cone-beam geometry, ray setup and sample positions (oracle).

Test infrastructure: only the tests, the smoke check and the benchmark's CPU legs
use it.

The paper renders X-rays whose source and detector positions are known
(Sec. 2.2) and samples points along each X-ray path (Sec. 2.1, Sec. 2.5), with
one view per batch, rays per view and points per ray as in Sec. 3.1. It does
not state the axis convention, the detector parametrisation or the sampling
rule; the readings used here are:

* volume: a cube of side ``vol_side_mm`` centred on the rotation axis, mapped to
  normalized coordinates x_hat in [0, 1]^3; every length below is in units of
  the cube side, so a unit-attenuation path of length one gives A = 1;
* source orbit about z: theta_v = angle0 + v * span / n_views,
  s = c0 + dso * (cos, sin, 0), detector centre = c0 - (dsd - dso) * (cos, sin, 0),
  detector axes u = (-sin, cos, 0), v = (0, 0, 1), c0 = (1/2, 1/2, 1/2);
* pixel (i, j) (pixel id = j * nu + i) sits at offsets ((i + 1/2) - nu/2) du and
  ((j + 1/2) - nv/2) dv from the detector centre;
* slab clipping against [0, 1]^3; a ray misses when near >= far;
* midpoint rule: t_i = near + (i + 1/2) Delta, Delta = (far - near) / N, and the
  step size of Eq. 1 is delta_i = Delta.

Per-view constants are computed in float64 and rounded once to float32. Every
per-ray and per-sample operation is then one correctly rounded float32
operation, in the order written, so the GPU (which spells the same sequence
with explicitly rounded intrinsics) reproduces positions bit for bit.
"""
from __future__ import annotations

import math

import numpy as np

f32 = np.float32


def view_table(n_views, angle0_rad, span_rad, dso_mm, dsd_mm, det_du_mm, det_dv_mm,
               vol_side_mm):
    """Per-view float32 table (V, 12): source s, detector centre c, axes u, v.

    Returns (table, du, dv) with du, dv the pixel pitches in volume units.
    """
    dso = dso_mm / vol_side_mm
    dsd = dsd_mm / vol_side_mm
    ddet = dsd - dso
    tab = np.zeros((n_views, 12), dtype=np.float32)
    for v in range(n_views):
        theta = angle0_rad + (v * span_rad) / n_views
        ct, st = math.cos(theta), math.sin(theta)
        row = [0.5 + dso * ct, 0.5 + dso * st, 0.5,
               0.5 - ddet * ct, 0.5 - ddet * st, 0.5,
               -st, ct, 0.0,
               0.0, 0.0, 1.0]
        tab[v] = np.array(row, dtype=np.float64).astype(np.float32)
    return tab, f32(det_du_mm / vol_side_mm), f32(det_dv_mm / vol_side_mm)


def ray_setup(tab, du, dv, nu, nv, view, pix):
    """Origin, unit direction and [near, far] of each ray (all float32).

    Returns (o (R,3), d (R,3), near (R,), far (R,), hit (R,) bool).
    """
    pix = np.asarray(pix, dtype=np.int64)
    s = tab[view, 0:3]
    c = tab[view, 3:6]
    u = tab[view, 6:9]
    v = tab[view, 9:12]
    i = (pix % nu).astype(np.float32)
    j = (pix // nu).astype(np.float32)
    half_nu = f32(nu) * f32(0.5)
    half_nv = f32(nv) * f32(0.5)
    ou = ((i + f32(0.5)) - half_nu) * f32(du)
    ov = ((j + f32(0.5)) - half_nv) * f32(dv)
    R = len(pix)
    d = np.zeros((R, 3), dtype=np.float32)
    for k in range(3):
        P = (c[k] + ou * u[k]) + ov * v[k]
        d[:, k] = P - s[k]
    len2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
    length = np.sqrt(len2)
    dn = (d / length[:, None]).astype(np.float32)
    near = np.zeros(R, dtype=np.float32)
    far = np.full(R, np.inf, dtype=np.float32)
    hit = np.ones(R, dtype=bool)
    with np.errstate(divide="ignore", invalid="ignore"):
        for k in range(3):
            dk = dn[:, k]
            nz = dk != 0
            ta = (f32(0.0) - s[k]) / dk
            tb = (f32(1.0) - s[k]) / dk
            t0 = np.minimum(ta, tb)
            t1 = np.maximum(ta, tb)
            near = np.where(nz, np.maximum(near, t0), near)
            far = np.where(nz, np.minimum(far, t1), far)
            outside = (s[k] < f32(0.0)) | (s[k] > f32(1.0))
            hit &= nz | ~outside
    hit &= near < far
    near = np.where(hit, near, f32(0.0)).astype(np.float32)
    far = np.where(hit, far, f32(0.0)).astype(np.float32)
    o = np.broadcast_to(s, (R, 3)).astype(np.float32)
    return o, dn, near, far, hit


def splitmix64(seed, k):
    """Output number k (k >= 1, uint64 array) of the SplitMix64 generator started at
    `seed` (Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
    2014): the state advances by the golden-ratio increment and is then mixed."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + np.uint64(0x9E3779B97F4A7C15) * np.asarray(k, dtype=np.uint64)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def stratum_offsets(seed, pix, N):
    """Offsets u (R, N) float32 of each sample inside its stratum: 1/2 when seed is 0
    (midpoint rule), else the top 24 bits of SplitMix64 output pix_r * N + i + 1
    times 2^-24 (stratified jitter; exact in float32)."""
    pix = np.asarray(pix)
    if seed == 0:
        return np.full((len(pix), N), f32(0.5), dtype=np.float32)
    k = (pix.astype(np.uint64)[:, None] * np.uint64(N) + np.arange(N, dtype=np.uint64)[None, :]
         + np.uint64(1))
    return (splitmix64(seed, k) >> np.uint64(40)).astype(np.float32) * f32(2.0 ** -24)


def sample_points(o, d, near, far, N, u=None):
    """Samples x_i = o + t_i d (float32, (R, N, 3)) and Delta (R,), with
    t_i = near + (i + u_i) Delta: the midpoint rule (u = 1/2) unless per-sample
    stratum offsets u (R, N) are given."""
    delta = (far - near) / f32(N)
    if u is None:
        ti = (np.arange(N, dtype=np.float32) + f32(0.5))[None, :]
    else:
        ti = np.arange(N, dtype=np.float32)[None, :] + np.asarray(u, dtype=np.float32)
    t = near[:, None] + ti * delta[:, None]
    x = o[:, None, :] + t[:, :, None] * d[:, None, :]
    return x.astype(np.float32), delta.astype(np.float32)


def voxel_centres_f32(D):
    """Voxel centres ((k + 1/2) / D in float32) of a D^3 grid, flattened [z][y][x] -> (D^3, 3)."""
    g = (np.arange(D, dtype=np.float32) + f32(0.5)) / f32(D)
    z, y, x = np.meshgrid(g, g, g, indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=-1).astype(np.float32)
