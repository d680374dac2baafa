"""Training at the tiny configuration (64^3 phantom, 50 views of 64^2, L8 F2 T2^14
16..64 with per-level normalization, 2x32 MLP, 1024 rays x 64 samples) in FP32,
BF16 and FP16 against the FP64 oracle's trajectory from the same initial
parameters and batches: the per-step loss error and the PSNR of the final field
(query at the 64^3 voxel centres against the phantom) are reported, and bounded by
each precision's tolerance.

The oracle's measurements are its own projections of the phantom (views used by
the batches only) with the seeded Poisson noise; the CUDA path receives the same
numbers."""
import dataclasses

import numpy as np
import pytest

import oracle
import synthetic as S
from _cases import hit_pixels, oracle_geom

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

W = S.WORKLOADS["tiny_fp32"]
STEPS = 10
# per-step relative loss error bound: FP32 (rounding amplified by Adam's
# normalisation of tiny gradients over the steps), and the mixed forms' forward
# tolerance (15 / 25 half-ulps of the 16-bit formats) doubled for the squared residual
LOSS_TOL = {S.PREC_F32: 1e-3, S.PREC_BF16: 2 * 15 * 2.0 ** -9, S.PREC_F16: 2 * 25 * 2.0 ** -12}


def _psnr(vol, ref):
    mse = float(np.mean((np.asarray(vol, np.float64) - ref) ** 2))
    return 10.0 * np.log10(1.0 / mse)


@pytest.fixture(scope="module")
def trajectory():
    og = oracle_geom(W.geometry)
    tab, du, dv, nu, nv = og
    vol, _ = S.phantom(W, 0)
    rng = np.random.default_rng(21)
    views = rng.integers(0, W.geometry.n_views, size=STEPS)
    used = sorted(set(views.tolist()))
    clean = oracle.project((tab[used], du, dv, nu, nv), vol, oversample=2)
    meas = S.poisson_measure(clean, W.I0, 22)
    batches = []
    for v in views:
        pix = rng.choice(hit_pixels(W.geometry, int(v)), size=W.n_rays, replace=False).astype(np.int32)
        batches.append((int(v), pix, meas[used.index(int(v))].ravel()[pix].astype(np.float32)))
    flat0 = S.init_params(W.field, 3).astype(np.float32)
    p, st = flat0.astype(np.float64), oracle.AdamState.zeros(flat0.size)
    losses = []
    for v, pix, a in batches:
        p, st, loss, _ = oracle.train_step(p, st, W.field, og, v, pix, a, W.n_samples)
        losses.append(loss)
    vol_ref = oracle.query_volume(p, W.field, W.vol_D)
    return batches, flat0, np.array(losses), _psnr(vol_ref, vol), vol


@pytest.mark.parametrize("precision", [S.PREC_F32, S.PREC_BF16, S.PREC_F16])
def test_training_in_each_precision_tracks_the_fp64_oracle(lib, trajectory, precision):
    batches, flat0, ref_losses, ref_psnr, vol = trajectory
    cfg = dataclasses.replace(W.field, precision=precision,
                              loss_scale_init=1024.0 if precision == S.PREC_F16 else 1.0)
    field = lib.Field(cfg, params=flat0)
    geom = lib.Geometry.from_config(W.geometry)
    ws = lib.workspace(lib.step_workspace_bytes(field, W.n_rays, W.n_samples))
    loss_t = torch.zeros(1, device="cuda")
    losses = []
    for v, pix, a in batches:
        lib.train_step(field, geom, v, torch.from_numpy(pix).cuda(), torch.from_numpy(a).cuda(), W.n_samples,
                       loss_t, ws)
        losses.append(float(loss_t.item()))
    flags, _, step = field.poll_status()
    assert flags == 0 and step == STEPS
    rel = np.abs(np.array(losses) - ref_losses) / ref_losses
    out = torch.empty(W.vol_D ** 3, device="cuda")
    lib.query_volume(field, W.vol_D, out)
    psnr = _psnr(out.cpu().numpy().reshape(vol.shape), vol)
    print(f"precision {precision}: per-step loss rel error max {rel.max():.2e} mean {rel.mean():.2e}; "
          f"final PSNR {psnr:.3f} dB vs oracle {ref_psnr:.3f} dB (delta {psnr - ref_psnr:+.4f})")
    assert rel.max() <= LOSS_TOL[precision], rel
    assert abs(psnr - ref_psnr) <= 0.1
