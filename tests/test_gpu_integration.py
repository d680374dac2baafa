"""Integration: the paper-scale configuration (128^3 textured phantom, 50 views of
256^2, L16 F2 T2^19 16..2048 with one LayerNorm, 4x32 MLP, 2048 rays x 192
samples) reconstructs. Trained through the library's kernels, FP32 and the mixed
BF16 path each pass 30 dB PSNR within 1000 steps. They end within 0.5 dB of each
other, and their 3-D SSIM is high."""
import numpy as np
import pytest

import synthetic as S

pytestmark = pytest.mark.gpu


def _scan(lib, torch, w, seed):
    geom = lib.Geometry.from_config(w.geometry)
    vol, _ = S.phantom(w, seed)
    D = vol.shape[0]
    g = w.geometry
    n = g.n_views * g.det_nv * g.det_nu
    proj = torch.empty(n, device="cuda")
    lib.project(geom, torch.from_numpy(vol.astype(np.float32)).cuda(), 2, proj)
    hitp = torch.empty(n, device="cuda")
    lib.project(geom, torch.ones(D ** 3, device="cuda"), 1, hitp)
    hit = hitp.view(g.n_views, -1).cpu().numpy() > 0
    a_meas = S.poisson_measure(proj.view(g.n_views, -1).cpu().numpy(), w.I0, seed + 1)
    cands = [np.nonzero(hit[v])[0] for v in range(g.n_views)]
    return geom, torch.from_numpy(vol.astype(np.float32).ravel()).cuda(), a_meas, cands


def test_paper_scale_training_reaches_30db_in_fp32_and_bf16(lib):
    import torch
    from paper_2506_19742_gb300 import recon
    final = {}
    for wname in ("paper_fp32", "paper_bf16"):
        w = S.WORKLOADS[wname]
        geom, vol_gt, a_meas, cands = _scan(lib, torch, w, 11)
        rec = recon.Reconstruction(w.field, geom, params=S.init_params(w.field, 0))
        rng = np.random.default_rng(12)
        psnr = {}
        for s in range(1, 1001):
            view, pix = S.pick_rays(rng, w.geometry.n_views, cands, w.n_rays)
            rec.step(view, torch.from_numpy(pix).cuda(), torch.from_numpy(a_meas[view][pix].astype(np.float32)).cuda(),
                     w.n_samples)
            if s % 250 == 0:
                psnr[s] = rec.psnr(vol_gt)
        flags, _, step = rec.field.poll_status()
        assert flags == 0 and step == 1000
        assert psnr[1000] >= 30.0, (wname, psnr)
        assert psnr[1000] > psnr[250] + 5.0, (wname, psnr)
        final[wname] = (psnr[1000], rec.ssim(vol_gt))
    assert abs(final["paper_bf16"][0] - final["paper_fp32"][0]) <= 0.5, final
    assert min(v[1] for v in final.values()) >= 0.9, final
