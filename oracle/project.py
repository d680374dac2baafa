"""Cone-beam forward projector (oracle), standing in for TIGRE (Sec. 3.1).

Test infrastructure: only the tests, the smoke check and the benchmark's CPU legs
use it.

The paper makes its projections with the TIGRE toolbox under the NAF setting
(Sec. 3.1). This stand-in integrates a voxel volume along the same rays as the
training sampler: for each detector pixel, the clipped ray [near, far] is cut
into n = ceil((far - near) * D * oversample) equal steps, the volume is
trilinearly interpolated at the step midpoints (voxel centres at (k + 1/2) / D,
zero outside the volume) and the line integral is the midpoint sum
sum_i vol(x_i) * Delta, the Beer-Lambert A of Eq. 1 for the voxel field.

Step counts, positions and interpolation fractions are float32 (mirrored with
the GPU); interpolation weights and the sum are float64.
"""
from __future__ import annotations

import numpy as np

from .geometry import ray_setup

f32 = np.float32


def project(geom, vol, oversample=2):
    """Projections (V, nv, nu) float64 of vol (D, D, D) [z][y][x] for every view of geom."""
    tab, du, dv, nu, nv = geom
    vol = np.asarray(vol, dtype=np.float64)
    D = vol.shape[0]
    V = tab.shape[0]
    out = np.zeros((V, nv, nu))
    pix = np.arange(nu * nv, dtype=np.int64)
    scale = f32(D * oversample)
    for view in range(V):
        o, d, near, far, hit = ray_setup(tab, du, dv, nu, nv, view, pix)
        n = np.where(hit, np.ceil((far - near) * scale), 0).astype(np.int64)
        nmax = int(n.max()) if n.size else 0
        if nmax == 0:
            continue
        delta = np.where(hit, (far - near) / np.maximum(n, 1).astype(np.float32), f32(0))
        delta = delta.astype(np.float32)
        A = np.zeros(len(pix))
        for i in range(nmax):
            live = i < n
            t = near + (f32(i) + f32(0.5)) * delta
            x = o + t[:, None] * d                          # (R, 3) float32
            pc = x * f32(D) - f32(0.5)
            i0 = np.floor(pc).astype(np.int64)
            fr = (pc - i0.astype(np.float32)).astype(np.float64)
            val = np.zeros(len(pix))
            for corner in range(8):
                b = np.array([(corner >> k) & 1 for k in range(3)])
                ii = i0 + b[None, :]
                w = np.prod(np.where(b[None, :] == 1, fr, 1.0 - fr), axis=1)
                ok = np.all((ii >= 0) & (ii < D), axis=1)
                iic = np.clip(ii, 0, D - 1)
                val += np.where(ok, w * vol[iic[:, 2], iic[:, 1], iic[:, 0]], 0.0)
            A += np.where(live, val * delta.astype(np.float64), 0.0)
        out[view] = A.reshape(nv, nu)
    return out
