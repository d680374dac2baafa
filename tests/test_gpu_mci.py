"""Mapping Consistency Initialization (Sec. 2.1, 2.4) on the GPU: an LN + MLP
pre-trained with the voxel loss (Eq. 2) on fields that the method itself
reconstructed starts new cases ahead of random initialisation.

Everything runs through the library's kernels (train_step, query_volume,
fit_points_step, field export / import); the control is the same case from the
same random hash tables and MLP initialisation without the transfer."""
import dataclasses

import numpy as np
import pytest

import synthetic as S

pytestmark = pytest.mark.gpu

# A reduced C2-shaped problem: 64^3 textured phantoms, 50 views of 96^2, L16 F2
# T2^16 16..512 with one LayerNorm, 4x32 MLP, 1024 rays x 96 samples.
GEOM = S.GeometryConfig(det_nu=96, det_nv=96)
FIELD = S.FieldConfig(n_levels=16, n_feat=2, log2_T=16, base_res=16, max_res=512, norm=S.NORM_LN,
                      hidden_layers=4, width=32)
WL = S.Workload("mci_small", 64, 8, True, False, GEOM, FIELD, 1024, 96, 0)


def _scan(nh, torch, seed):
    geom = nh.Geometry.from_config(GEOM)
    vol, _ = S.phantom(WL, seed)
    D = vol.shape[0]
    nproj = GEOM.n_views * GEOM.det_nv * GEOM.det_nu
    proj = torch.empty(nproj, device="cuda")
    nh.project(geom, torch.from_numpy(vol.astype(np.float32)).cuda(), 2, proj)
    hitp = torch.empty(nproj, device="cuda")
    nh.project(geom, torch.ones(D ** 3, device="cuda"), 1, hitp)
    clean = proj.view(GEOM.n_views, -1).cpu().numpy()
    hit = hitp.view(GEOM.n_views, -1).cpu().numpy() > 0
    a_meas = S.poisson_measure(clean, WL.I0, seed + 1)
    cands = [np.nonzero(hit[v])[0] for v in range(GEOM.n_views)]
    return geom, torch.from_numpy(vol.astype(np.float32).ravel()).cuda(), a_meas, cands


def _train(nh, torch, recon, scan, seed, steps, checkpoints, ln_mlp=None):
    geom, vol_gt, a_meas, cands = scan
    rec = recon.Reconstruction(FIELD, geom, params=S.init_params(FIELD, seed))
    if ln_mlp is not None:
        recon.transfer(ln_mlp, rec.field)
    rng = np.random.default_rng(seed + 7)
    psnr = {}
    for s in range(1, steps + 1):
        view, pix = S.pick_rays(rng, GEOM.n_views, cands, WL.n_rays)
        rec.step(view, torch.from_numpy(pix).cuda(),
                 torch.from_numpy(a_meas[view][pix].astype(np.float32)).cuda(), WL.n_samples)
        if s in checkpoints:
            psnr[s] = rec.psnr(vol_gt)
    return rec, psnr


def test_mci_pretrained_ln_mlp_starts_ahead_of_random_init(lib):
    torch = pytest.importorskip("torch")
    from paper_2506_19742_gb300 import nhcbct as nh
    from paper_2506_19742_gb300 import recon

    # 1. reconstruct three pre-training cases with the method itself
    vols = []
    for seed in (100, 101, 102):
        rec, p = _train(nh, torch, recon, _scan(nh, torch, seed), seed, 400, {400})
        assert p[400] > 24.0, p
        vols.append(rec.volume(64))
    # 2. fit one shared LN + MLP to the reconstructions (Eq. 2), per-case hash tables
    shared, curve = recon.pretrain_mci(FIELD, vols, steps=600, points_per_step=32768, seed=3)
    assert curve[-1][1] < curve[0][1]
    assert shared.numel() == nh.Field(FIELD).export_bytes(recon.LN_MLP) // 4
    # 3. held-out cases: random initialisation vs the same initialisation + transfer
    gains = []
    for seed in (200, 201):
        scan = _scan(nh, torch, seed)
        _, pr = _train(nh, torch, recon, scan, seed, 100, {25, 50, 100})
        _, pm = _train(nh, torch, recon, scan, seed, 100, {25, 50, 100}, ln_mlp=shared)
        print(f"seed {seed}: random {pr}  mci {pm}")
        gains.append(pm[50] - pr[50])
    assert np.mean(gains) > 1.0, gains
