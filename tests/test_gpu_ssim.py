"""3-D SSIM on the GPU (ssim3d) against the oracle: the local index at every
window position and the mean, on random and phantom volumes, from a single window
(D = 11) through ragged sizes to the 128^3 read-out grid of the paper workload."""
import numpy as np
import pytest

import oracle
import synthetic as S

pytestmark = pytest.mark.gpu


def _pair(D, seed, noise=0.15):
    rng = np.random.default_rng(seed)
    x = rng.random((D, D, D)).astype(np.float32)
    y = np.clip(0.7 * x + 0.15 + noise * rng.standard_normal((D, D, D)), 0.0, 1.0).astype(np.float32)
    return x, y


@pytest.mark.parametrize("D", [11, 12, 23, 37])
def test_ssim_map_and_mean_match_the_oracle(lib, D):
    import torch
    x, y = _pair(D, D)
    M = D - 10
    got_map = torch.empty(M ** 3, dtype=torch.float64, device="cuda")
    got = lib.ssim3d(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(), map_out=got_map)
    torch.cuda.synchronize()
    want_map = oracle.ssim_map(x, y)
    np.testing.assert_allclose(got_map.cpu().numpy().reshape(M, M, M), want_map, rtol=0, atol=1e-10)
    assert abs(float(got.item()) - float(want_map.mean())) < 1e-11
    # a repeated call gives the same bits (fixed summation order)
    again = lib.ssim3d(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda())
    assert float(again.item()) == float(got.item())


def test_ssim_identical_volumes_and_data_range(lib):
    import torch
    x, y = _pair(16, 1)
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    assert abs(lib.ssim(xd, xd) - 1.0) < 1e-12
    got = lib.ssim3d(xd, yd, data_range=2.0)
    assert abs(float(got.item()) - oracle.ssim(x, y, data_range=2.0)) < 1e-11


def test_ssim_at_the_paper_read_out_grid(lib):
    """128^3 textured phantom against a noisy copy (the size the view sweep scores):
    sampled window positions against the oracle on their own 11^3 cube, the mean
    against the mean of the returned map, identical volumes score 1."""
    import torch
    w = S.WORKLOADS["paper_fp32"]
    vol, _ = S.phantom(w, 7)
    x = vol.astype(np.float32)
    D = x.shape[0]
    assert D == 128
    y = np.clip(x + 0.05 * np.random.default_rng(8).standard_normal(x.shape), 0.0, 1.0).astype(np.float32)
    M = D - 10
    got_map = torch.empty(M ** 3, dtype=torch.float64, device="cuda")
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    got = float(lib.ssim3d(xd, yd, map_out=got_map).item())
    gm = got_map.cpu().numpy().reshape(M, M, M)
    rng = np.random.default_rng(9)
    pos = [(0, 0, 0), (M - 1, M - 1, M - 1), (M // 2, 3, M - 2)] + [tuple(p) for p in rng.integers(0, M, (61, 3))]
    for z, yy, xx in pos:
        want = oracle.ssim_map(x[z:z + 11, yy:yy + 11, xx:xx + 11], y[z:z + 11, yy:yy + 11, xx:xx + 11])
        assert abs(gm[z, yy, xx] - want[0, 0, 0]) < 1e-10, (z, yy, xx)
    assert abs(got - gm.mean()) < 1e-12
    assert 0.0 < got < 1.0
    assert abs(lib.ssim(xd, xd) - 1.0) < 1e-12
