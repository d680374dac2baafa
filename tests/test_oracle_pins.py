"""Pins for the CPU oracle: closed forms, library routines, brute force and finite
differences. None of these re-type the oracle's own formulas; each is chosen so a
plausible slip (a dropped term, a wrong sign or index, a transposed operand) fails."""
import dataclasses
import math

import numpy as np
import pytest

import oracle
import synthetic as S
from _cases import C4_SUB, C4_SUB_N, c4_subinstance

TINY_F = S.FieldConfig(n_levels=2, n_feat=2, log2_T=8, base_res=2, max_res=8,
                       norm=S.NORM_LN, hidden_layers=2, width=8)


def _geom(g: S.GeometryConfig):
    tab, du, dv = oracle.view_table(g.n_views, g.angle0_rad, g.span_rad, g.dso_mm, g.dsd_mm,
                                    g.det_du_mm, g.det_dv_mm, g.vol_side_mm)
    return (tab, du, dv, g.det_nu, g.det_nv)


def _box_chord64(o, d):
    """Exact chord of the ray o + t d (float64) through [0,1]^3 (0 on a miss)."""
    lo, hi = -np.inf, np.inf
    for k in range(3):
        if d[k] == 0.0:
            if not (0.0 <= o[k] <= 1.0):
                return 0.0
            continue
        a, b = (0.0 - o[k]) / d[k], (1.0 - o[k]) / d[k]
        lo, hi = max(lo, min(a, b)), min(hi, max(a, b))
    lo = max(lo, 0.0)
    return max(hi - lo, 0.0)


# ---------------------------------------------------------------- encoding
@pytest.mark.parametrize("L,base,top", [(8, 16, 64), (16, 16, 2048), (4, 3, 17), (1, 5, 5)])
def test_level_resolutions_integer_bracket(L, base, top):
    """N_l = floor(base (top/base)^(l/(L-1))), checked in exact integer arithmetic:
    N^(L-1) <= base^(L-1-l) top^l < (N+1)^(L-1)."""
    res = oracle.level_resolutions(L, base, top)
    assert res[0] == base and res[-1] == top
    if L == 1:
        return
    for l, n in enumerate(res):
        target = base ** (L - 1 - l) * top ** l
        assert n ** (L - 1) <= target < (n + 1) ** (L - 1), (l, n)


def test_level_resolutions_named_workloads():
    assert oracle.level_resolutions(8, 16, 64) == [16, 19, 23, 28, 35, 43, 52, 64]
    assert oracle.level_resolutions(16, 16, 2048) == [16, 22, 30, 42, 58, 80, 111, 153, 212,
                                                      294, 406, 561, 776, 1072, 1482, 2048]


def test_dense_level_is_a_bijection():
    """Every vertex of a dense level gets its own entry in [0, (N+1)^3)."""
    n, T = 7, 1 << 9
    g = (np.arange(n + 1) / n).astype(np.float32)
    X = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    idx, w, _ = oracle.corners(X * np.float32(0.999), [n], T)   # cell origin = vertex below
    verts = set()
    for corner in range(8):
        verts |= set(idx[:, 0, corner].tolist())
    assert verts == set(range((n + 1) ** 3))


def test_hashed_level_special_cases_and_spread():
    """With the x prime equal to 1, points on the x axis map to cx mod T; on the y
    and z axes the index is (c * pi) mod 2^32 mod T with the published per-axis
    primes pi_2 = 2654435761 and pi_3 = 805459861 of the spatial hash (Teschner et
    al. 2003, as used by Mueller et al. 2022), computed here in exact integers; the
    index stays below T; buckets of a large random sample are roughly uniform."""
    n, T = 512, 1 << 10
    x = np.zeros((n, 3), dtype=np.float32)
    x[:, 0] = (np.arange(n, dtype=np.float32) + np.float32(0.25)) / np.float32(n)
    idx, _, _ = oracle.corners(x, [n], T)
    assert np.array_equal(idx[:, 0, 0], np.arange(n) % T)
    assert np.array_equal(idx[:, 0, 1], (np.arange(n) + 1) % T)
    for axis, prime in ((1, 2654435761), (2, 805459861)):
        xa = np.zeros((n, 3), dtype=np.float32)
        xa[:, axis] = x[:, 0]
        idx, _, _ = oracle.corners(xa, [n], T)
        expect = [((c * prime) % (1 << 32)) % T for c in range(n)]
        assert idx[:, 0, 0].tolist() == expect
    rng = np.random.default_rng(0)
    xr = rng.random((20000, 3)).astype(np.float32)
    idx, _, _ = oracle.corners(xr, [n], T)
    assert idx.max() < T
    counts = np.bincount(idx[:, 0, :].ravel(), minlength=T)
    expect = counts.sum() / T
    chi2 = np.sum((counts - expect) ** 2 / expect)
    assert chi2 < 1.3 * T    # dof = T - 1; a biased hash lands far above


def test_trilinear_reproduces_linear_field_and_partition_of_unity():
    """On a collision-free dense level holding a linear function of the vertex
    coordinates, interpolation returns the same linear function of x_hat * N."""
    n, T = 8, 1 << 10
    F = 2
    a = np.array([[0.3, -1.2, 0.7], [2.0, 0.5, -0.25]])
    b = np.array([0.1, -0.4])
    table = np.zeros((1, T, F))
    for z in range(n + 1):
        for y in range(n + 1):
            for x in range(n + 1):
                i = x + y * (n + 1) + z * (n + 1) ** 2
                table[0, i] = a @ np.array([x, y, z]) + b
    rng = np.random.default_rng(3)
    pts = rng.random((500, 3)).astype(np.float32)
    pts[:5] = [[0, 0, 0], [1, 1, 1], [1, 0, 0.5], [0.999999, 0.5, 0], [0.125, 0.25, 0.375]]
    h = oracle.encode(pts, table, [n], T)
    ref = (pts.astype(np.float64) * n) @ a.T + b
    np.testing.assert_allclose(h, ref, rtol=0, atol=1e-12)
    _, w, _ = oracle.corners(pts, [n, 5, 64], 1 << 8)
    np.testing.assert_allclose(w.sum(axis=-1), 1.0, rtol=0, atol=1e-14)


# ---------------------------------------------------------------- geometry / sampler
def test_view_table_geometry():
    g = S.GeometryConfig(n_views=8, det_nu=16, det_nv=12)
    tab, du, dv, _, _ = _geom(g)
    c0 = np.array([0.5, 0.5, 0.5])
    for v in range(8):
        s, c, u, w = tab[v, :3], tab[v, 3:6], tab[v, 6:9], tab[v, 9:12]
        theta = 2 * math.pi * v / 8
        assert abs(np.linalg.norm(s - c0) - 1000 / 256) < 1e-5
        assert abs(np.linalg.norm(c - c0) - 500 / 256) < 1e-5
        assert abs(np.linalg.norm(s - c) - 1500 / 256) < 1e-5
        assert abs(np.dot(u, s - c)) < 1e-5 and abs(np.dot(w, s - c)) < 1e-5
        assert abs(math.atan2(s[1] - 0.5, s[0] - 0.5) % (2 * math.pi) - theta % (2 * math.pi)) < 1e-5 \
            or abs(abs(math.atan2(s[1] - 0.5, s[0] - 0.5) - theta) - 2 * math.pi) < 1e-5
    assert abs(du - 700 / 16 / 256) < 1e-7 and abs(dv - 700 / 12 / 256) < 1e-7


def test_ray_clip_matches_exact_box_chord_and_samples_are_midpoints():
    g = S.GeometryConfig(n_views=5, det_nu=24, det_nv=20)
    geom = _geom(g)
    tab, du, dv, nu, nv = geom
    pix = np.arange(nu * nv)
    N = 7
    for view in range(5):
        o, d, near, far, hit = oracle.ray_setup(tab, du, dv, nu, nv, view, pix)
        assert o.dtype == np.float32 and d.dtype == np.float32 and near.dtype == np.float32
        assert 0 < hit.sum() < len(pix)
        x, delta = oracle.sample_points(o, d, near, far, N)
        assert x.dtype == np.float32
        for r in range(len(pix)):
            chord = _box_chord64(o[r].astype(np.float64), d[r].astype(np.float64))
            if hit[r]:
                assert abs((far[r] - near[r]) - chord) < 2e-6
                assert abs(np.linalg.norm(d[r].astype(np.float64)) - 1) < 1e-6
                xs = x[r].astype(np.float64)
                assert np.all(xs > -1e-6) and np.all(xs < 1 + 1e-6)
                # equal spacing delta, first sample half a step past the entry point
                steps = np.linalg.norm(np.diff(xs, axis=0), axis=1)
                np.testing.assert_allclose(steps, delta[r], rtol=0, atol=1e-6)  # FP32 rounding at |s| ~ 4.4
                entry = o[r].astype(np.float64) + near[r] * d[r].astype(np.float64)
                assert abs(np.linalg.norm(xs[0] - entry) - 0.5 * delta[r]) < 1e-5
            else:
                assert chord < 1e-6


def test_detector_symmetry():
    """On an odd-sized detector the central pixel's ray passes through the rotation
    axis at the cube centre, and pixels mirrored about the detector centre see
    mirror-image rays with equal chords (left-right needs a view angle that is a
    multiple of 45 degrees, where the cube is mirror-symmetric too)."""
    g = S.GeometryConfig(n_views=8, det_nu=11, det_nv=9)
    tab, du, dv, nu, nv = _geom(g)
    pix = np.arange(nu * nv)
    for view in range(8):
        o, d, near, far, hit = oracle.ray_setup(tab, du, dv, nu, nv, view, pix)
        centre = (nv // 2) * nu + nu // 2
        oc, dc = o[centre].astype(np.float64), d[centre].astype(np.float64)
        dist = np.linalg.norm(np.cross(np.array([0.5, 0.5, 0.5]) - oc, dc))
        assert dist < 1e-6
        chord = (far - near).reshape(nv, nu).astype(np.float64)
        np.testing.assert_allclose(chord, chord[:, ::-1], atol=2e-6)
        np.testing.assert_allclose(chord, chord[::-1, :], atol=2e-6)


def test_voxel_read_out_grid_is_centred_and_x_fastest():
    """The read-out grid of query_volume / PSNR: D^3 voxels tiling [0, 1]^3, so the
    points lie symmetric about the volume centre with spacing 1/D, half a voxel in
    from each face, in [z][y][x] order (x varies fastest)."""
    for D in (1, 2, 5, 64):
        c = oracle.voxel_centres_f32(D).astype(np.float64)
        assert c.shape == (D ** 3, 3)
        np.testing.assert_allclose(c.mean(axis=0), 0.5, rtol=0, atol=1e-6)
        np.testing.assert_allclose(c + c[::-1], 1.0, rtol=0, atol=1e-6)   # point reflection through the centre
        np.testing.assert_allclose(c.min(axis=0), 0.5 / D, rtol=0, atol=1e-7)
        if D > 1:
            np.testing.assert_allclose(c[1, 0] - c[0, 0], 1.0 / D, rtol=0, atol=1e-6)
            np.testing.assert_allclose(c[D, 1] - c[0, 1], 1.0 / D, rtol=0, atol=1e-6)
            np.testing.assert_allclose(c[D * D, 2] - c[0, 2], 1.0 / D, rtol=0, atol=1e-6)


def test_constant_field_gives_c_times_chord():
    """mu == c everywhere (output weights 0, bias logit(c)) turns Eq. 1 into c * chord."""
    g = S.GeometryConfig(n_views=3, det_nu=16, det_nv=16)
    geom = _geom(g)
    tab, du, dv, nu, nv = geom
    p = oracle.unflatten(S.init_params(TINY_F, 1).astype(np.float64), TINY_F)
    c = 0.37
    p["W"][-1][:] = 0.0
    p["b"][-1][:] = math.log(c / (1 - c))
    flat = oracle.flatten(p)
    pix = np.arange(nu * nv)
    A = oracle.render(flat, TINY_F, geom, 1, pix, 33)
    o, d, near, far, hit = oracle.ray_setup(tab, du, dv, nu, nv, 1, pix)
    chords = np.array([_box_chord64(o[r].astype(np.float64), d[r].astype(np.float64))
                       for r in range(len(pix))])
    np.testing.assert_allclose(A, c * chords, rtol=0, atol=2e-6)
    assert np.all(A[~hit] == 0.0)


# ---------------------------------------------------------------- normalization and MLP
@pytest.mark.parametrize("norm", [S.NORM_LN, S.NORM_LN_PER_LEVEL])
def test_layer_norm_moments_and_torch(norm):
    torch = pytest.importorskip("torch")
    cfg = dataclasses.replace(TINY_F, n_levels=4, n_feat=4, norm=norm)
    D = 16
    rng = np.random.default_rng(5)
    h = rng.normal(size=(64, D)) * rng.uniform(1e-3, 2, size=(64, 1))
    gamma, beta = np.ones(D), np.zeros(D)
    y, (hhat, rstd) = oracle.normalize_forward(h, gamma, beta, np.ones(D), cfg)
    G = 1 if norm == S.NORM_LN else 4
    hg = h.reshape(64, G, D // G)
    var = hg.var(axis=-1)
    yg = y.reshape(64, G, D // G)
    np.testing.assert_allclose(yg.mean(axis=-1), 0, atol=1e-12)
    np.testing.assert_allclose(yg.var(axis=-1), var / (var + cfg.ln_eps), rtol=1e-10)
    gamma, beta = rng.normal(size=D), rng.normal(size=D)
    mask = (rng.random(D) > 0.3).astype(np.float64)
    y, _ = oracle.normalize_forward(h, gamma, beta, mask, cfg)
    ht = torch.tensor(hg, dtype=torch.float64)
    ref = torch.nn.functional.layer_norm(ht, (D // G,), eps=cfg.ln_eps).reshape(64, D).numpy()
    np.testing.assert_allclose(y, (ref * gamma + beta) * mask, rtol=1e-12, atol=1e-12)


def test_mlp_forward_matches_torch_modules():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(6)
    dims = [16, 32, 32, 32, 1]
    Ws = [rng.normal(size=(dims[k + 1], dims[k])) / 4 for k in range(4)]
    bs = [rng.normal(size=dims[k + 1]) / 4 for k in range(4)]
    y = rng.normal(size=(50, 16))
    mu, acts, zs = oracle.mlp_forward(y, Ws, bs)
    layers = []
    for k in range(4):
        lin = torch.nn.Linear(dims[k], dims[k + 1]).double()
        lin.weight.data = torch.tensor(Ws[k]); lin.bias.data = torch.tensor(bs[k])
        layers += [lin, torch.nn.ReLU() if k < 3 else torch.nn.Sigmoid()]
    ref = torch.nn.Sequential(*layers)(torch.tensor(y)).detach().numpy()[:, 0]
    np.testing.assert_allclose(mu, ref, rtol=1e-13)


# ---------------------------------------------------------------- gradients
def _tiny_setup(cfg, seed=0, table_scale=0.5):
    g = S.GeometryConfig(n_views=4, det_nu=8, det_nv=8)
    geom = _geom(g)
    tab, du, dv, nu, nv = geom
    rng = np.random.default_rng(seed)
    flat = S.init_params(cfg, seed, table_scale=table_scale).astype(np.float64)
    o, d, near, far, hit = oracle.ray_setup(tab, du, dv, nu, nv, 2, np.arange(nu * nv))
    pix = rng.choice(np.nonzero(hit)[0], size=6, replace=False).astype(np.int32)
    pix = np.concatenate([pix, np.nonzero(~hit)[0][:1]]).astype(np.int32)   # one miss
    A_meas = rng.uniform(0.0, 0.6, size=len(pix))
    return geom, flat, pix, A_meas


def _fd_check(fun, flat, grad, rng, n_pick=300, h=1e-6, tol=1e-6):
    nz = np.nonzero(grad)[0]
    pick = np.concatenate([rng.choice(nz, size=min(n_pick, len(nz)), replace=False),
                           rng.choice(len(flat), size=20, replace=False)])
    for i in pick:
        e = np.zeros_like(flat); e[i] = h * max(1.0, abs(flat[i]))
        fd = (fun(flat + e) - fun(flat - e)) / (2 * e[i])
        scale = max(1e-3, np.abs(grad).max())
        assert abs(fd - grad[i]) <= tol * scale + 1e-7 * abs(grad[i]), (i, fd, grad[i])


@pytest.mark.parametrize("norm", [S.NORM_NONE, S.NORM_LN, S.NORM_LN_PER_LEVEL])
def test_render_gradient_finite_differences(norm):
    """Central differences of the MSE pixel loss on a tiny instance with a dense and a
    hashed level (T = 2^8, forced collisions) agree with the analytic backward."""
    cfg = dataclasses.replace(TINY_F, norm=norm)
    geom, flat, pix, A_meas = _tiny_setup(cfg)
    mask = np.array([1.0, 0.0, 1.0, 1.0])
    N = 9

    def loss(fl):
        A = oracle.render(fl, cfg, geom, 2, pix, N, mask)
        return oracle.loss_and_grad(A, A_meas, S.LOSS_MSE)[0]

    A, cache = oracle.render_forward(flat, cfg, geom, 2, pix, N, mask)
    _, dLdA = oracle.loss_and_grad(A, A_meas, S.LOSS_MSE)
    grad = oracle.render_backward(cache, dLdA, cfg)
    _fd_check(loss, flat, grad, np.random.default_rng(1))


def test_render_gradient_finite_differences_c4_subinstance():
    """The backward (Sec. 2.5 training, Eq. 1 ray sum, LN, MLP, hash scatter with
    collisions) agrees with central differences at the large configuration's field
    shape."""
    geom, flat, pix, A_meas = c4_subinstance()
    N = C4_SUB_N
    assert oracle.level_resolutions(16, 16, 2048)[-1] == 2048

    def loss(fl):
        return oracle.loss_and_grad(oracle.render(fl, C4_SUB, geom, 1, pix, N), A_meas, S.LOSS_MSE)[0]

    A, cache = oracle.render_forward(flat, C4_SUB, geom, 1, pix, N)
    assert A[-1] == 0.0 and np.all(A[:-1] != 0.0)
    _, dLdA = oracle.loss_and_grad(A, A_meas, S.LOSS_MSE)
    grad = oracle.render_backward(cache, dLdA, C4_SUB)
    _fd_check(loss, flat, grad, np.random.default_rng(4), n_pick=200)


def test_l1_pixel_loss_and_voxel_loss_gradients():
    """Eq. 3 (L1) and Eq. 2 (voxel L1): FD of the loss matches the backward away from kinks."""
    cfg = dataclasses.replace(TINY_F, loss=S.LOSS_L1)
    geom, flat, pix, A_meas = _tiny_setup(cfg, seed=4)
    N = 5

    def loss(fl):
        A = oracle.render(fl, cfg, geom, 2, pix, N)
        return oracle.loss_and_grad(A, A_meas, S.LOSS_L1)[0]

    A, cache = oracle.render_forward(flat, cfg, geom, 2, pix, N)
    l1, dLdA = oracle.loss_and_grad(A, A_meas, S.LOSS_L1)
    assert abs(l1 - np.mean(np.abs(A - A_meas))) < 1e-15
    grad = oracle.render_backward(cache, dLdA, cfg)
    _fd_check(loss, flat, grad, np.random.default_rng(2))

    rng = np.random.default_rng(9)
    xyz = rng.random((40, 3)).astype(np.float32)
    mu_gt = rng.random(40)
    st = oracle.AdamState.zeros(flat.size)
    _, _, vloss, vgrad = oracle.fit_points_step(flat, st, cfg, xyz, mu_gt, adam=False)
    mu = oracle.query_points(flat, cfg, xyz)
    assert abs(vloss - np.mean(np.abs(mu_gt - mu))) < 1e-15
    _fd_check(lambda fl: np.mean(np.abs(mu_gt - oracle.query_points(fl, cfg, xyz))),
              flat, vgrad, np.random.default_rng(3))


def test_losses_special_values():
    A = np.array([0.5, 1.0, 2.0])
    Am = np.array([0.5, 0.0, 3.0])
    l, g = oracle.loss_and_grad(A, Am, S.LOSS_MSE)
    assert abs(l - (0 + 1 + 1) / 3) < 1e-15
    np.testing.assert_allclose(g, [0, 2 / 3, -2 / 3])
    l, g = oracle.loss_and_grad(A, Am, S.LOSS_L1)
    assert abs(l - 2 / 3) < 1e-15
    np.testing.assert_allclose(g, [0, 1 / 3, -1 / 3])


# ---------------------------------------------------------------- Adam
def test_adam_matches_torch_optim():
    torch = pytest.importorskip("torch")
    cfg = TINY_F
    rng = np.random.default_rng(7)
    p0 = rng.normal(size=50)
    st = oracle.AdamState.zeros(50)
    pt = torch.tensor(p0.copy(), requires_grad=True)
    opt = torch.optim.Adam([pt], lr=cfg.lr, betas=(cfg.beta1, cfg.beta2), eps=cfg.adam_eps)
    p = p0.copy()
    for step in range(4):
        g = rng.normal(size=50) * (10.0 ** -step)
        g[:5] = 0.0                         # untouched entries still decay their moments
        p, st, skipped = oracle.adam_step(p, g * 8.0, st, cfg, loss_scale=8.0)
        assert not skipped
        pt.grad = torch.tensor(g)
        opt.step()
        np.testing.assert_allclose(p, pt.detach().numpy(), rtol=1e-12, atol=1e-15)
    g = np.full(50, np.inf)
    p2, st2, skipped = oracle.adam_step(p, g, st, cfg)
    assert skipped and st2.t == st.t and np.array_equal(p2, p)


def test_adam_leaves_zero_gradient_zero_moment_entries_bit_for_bit():
    # the step of an entry whose gradient and moments are zero is exactly zero:
    # m = v = 0 give lr * 0 / (0 + eps), so p comes back with the same bits, at
    # every step count (the bias corrections multiply zeros)
    cfg = TINY_F
    rng = np.random.default_rng(11)
    p = rng.normal(size=64)
    p0 = p.copy()
    st = oracle.AdamState.zeros(64)
    for step in range(5):
        g = rng.normal(size=64)
        g[:16] = 0.0
        p, st, _ = oracle.adam_step(p, g, st, cfg)
    assert np.array_equal(p[:16], p0[:16])
    assert not np.any(st.m[:16]) and not np.any(st.v[:16])
    assert not np.array_equal(p[16:], p0[16:])


def test_dense_levels_give_no_gradient_past_their_grid_vertices():
    # a dense level (N_l + 1)^3 <= T indexes corner (x, y, z) at x + y (N + 1) +
    # z (N + 1)^2 <= (N + 1)^3 - 1, so the backward never reaches its later entries
    # (the optimizer may skip them); the hashed levels' entries are all reachable
    from _cases import batch, field_cfg, oracle_geom
    from oracle.encoding import is_dense, level_resolutions
    cfg = field_cfg(n_levels=8, log2_T=12, base_res=4, max_res=48)
    geom = S.GeometryConfig(n_views=6, det_nu=40, det_nv=36)
    flat = S.init_params(cfg, 3, table_scale=0.5).astype(np.float64)
    pix = batch(geom, 2, 150, seed=1)
    A, cache = oracle.render_forward(flat, cfg, oracle_geom(geom), 2, pix, 24)
    _, dLdA = oracle.loss_and_grad(A, np.zeros(len(pix)), S.LOSS_MSE)
    g = oracle.render_backward(cache, dLdA, cfg)
    T, F = 2 ** cfg.log2_T, cfg.n_feat
    dense = 0
    for l, res in enumerate(level_resolutions(cfg.n_levels, cfg.base_res, cfg.max_res)):
        lev = g[l * T * F:(l + 1) * T * F]
        if is_dense(res, T):
            dense += 1
            n_l = (res + 1) ** 3
            assert not np.any(lev[n_l * F:]), (l, res)
            assert np.any(lev[:n_l * F])
    assert dense >= 3


# ---------------------------------------------------------------- projector
def _ellipsoid_chord(o, d, E):
    """Exact line integral of a top-index-wins ellipsoid phantom along o + t d (t >= 0),
    from the sorted chord endpoints of every ellipsoid (volume units, cube [0,1]^3)."""
    ts = []
    spans = []
    for k in range(len(E.values)):
        c = E.centres[k] + 0.5
        A0 = ((o - c) @ E.rot[k]) / E.axes[k]
        B0 = (d @ E.rot[k]) / E.axes[k]
        qa, qb, qc = B0 @ B0, 2 * A0 @ B0, A0 @ A0 - 1
        disc = qb * qb - 4 * qa * qc
        if disc <= 0:
            spans.append(None)
            continue
        t1 = (-qb - math.sqrt(disc)) / (2 * qa)
        t2 = (-qb + math.sqrt(disc)) / (2 * qa)
        spans.append((t1, t2))
        ts += [t1, t2]
    ts = sorted(ts)
    total = 0.0
    for a, b in zip(ts[:-1], ts[1:]):
        mid = 0.5 * (a + b)
        val = 0.0
        for k, sp in enumerate(spans):
            if sp is not None and sp[0] <= mid <= sp[1]:
                val = E.values[k]
        total += val * (b - a)
    return total


def test_projector_converges_to_analytic_ellipsoid_integrals():
    g = S.GeometryConfig(n_views=2, det_nu=12, det_nv=12)
    geom = _geom(g)
    tab, du, dv, nu, nv = geom
    E = S.random_ellipsoids(3, seed=11)
    pix = np.arange(nu * nv)
    exact = np.zeros((2, nv, nu))
    for view in range(2):
        o, d, near, far, hit = oracle.ray_setup(tab, du, dv, nu, nv, view, pix)
        for r in range(len(pix)):
            if hit[r]:
                exact[view].flat[r] = _ellipsoid_chord(o[r].astype(np.float64),
                                                       d[r].astype(np.float64), E)
    errs = []
    for D in (16, 32, 64):
        vol = S.paint_ellipsoids(E, D)
        proj = oracle.project(geom, vol, oversample=2)
        errs.append(np.mean(np.abs(proj - exact)))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 0.1 * np.mean(np.abs(exact)) and exact.max() > 0.02


def test_projector_of_uniform_volume_is_chord_less_boundary_ramp():
    """Ones inside the cube, zero outside. Between a face and the first voxel centre
    the trilinear value ramps linearly from 1/2 to 1, which costs exactly
    1/(8 D |d_k|) of path integral per face of axis k crossed: a ray along x through
    the interior loses 1/(4 D |d_x|), and no ray loses more than sum_k 1/(4 D |d_k|)."""
    g = S.GeometryConfig(n_views=2, det_nu=10, det_nv=10)
    geom = _geom(g)
    tab, du, dv, nu, nv = geom
    D = 16
    proj = oracle.project(geom, np.ones((D, D, D)), oversample=8)
    for view in range(2):
        o, d, near, far, hit = oracle.ray_setup(tab, du, dv, nu, nv, view, np.arange(nu * nv))
        chord = (far - near).astype(np.float64)
        loss = chord - proj[view].ravel()
        assert np.all(loss >= -1e-6)
        ad = np.abs(d.astype(np.float64))
        with np.errstate(divide="ignore"):
            bound = np.minimum(1.0 / (4 * D * ad), chord[:, None] / 2).sum(axis=1)
        assert np.all(loss[hit] <= bound[hit] + 1e-4)
        centre = (nv // 2) * nu + nu // 2
        axis = int(np.argmax(ad[centre]))
        assert abs(loss[centre] - 1.0 / (4 * D * ad[centre, axis])) < 2e-4


# ---------------------------------------------------------------- FFT channel masking (Sec. 2.3)
def test_fft_high_frequency_fraction_of_tones_constants_and_white_noise():
    """Pure tones put all their power at one radius |k| = |n| / G, a constant has
    none, and white noise spreads it evenly over the G^3 - 1 non-zero bins. The
    statistic is taken on each channel's mean-free spectrum, so a constant offset
    added to a tone leaves its fraction unchanged."""
    G = 16
    z, y, x = np.meshgrid(np.arange(G), np.arange(G), np.arange(G), indexing="ij")
    noise = np.random.default_rng(0).normal(size=(G, G, G))
    chans = [np.cos(2 * np.pi * 2 * x / G),            # |k| = 0.125
             np.cos(2 * np.pi * 6 * y / G),            # |k| = 0.375
             np.sin(2 * np.pi * (3 * x + 3 * z) / G),  # |k| = 3 sqrt(2) / 16 = 0.265
             np.full((G, G, G), 0.7), noise, np.cos(2 * np.pi * 6 * y / G) + 5.0]
    h = np.stack(chans, axis=-1).reshape(G ** 3, -1)
    frac = oracle.high_frequency_fraction(h, G, 0.25)
    np.testing.assert_allclose(frac[:4], [0.0, 1.0, 1.0, 0.0], atol=1e-12)
    assert abs(frac[5] - 1.0) < 1e-12
    n_high = sum(1 for a in range(-G // 2, G // 2) for b in range(-G // 2, G // 2)
                 for c in range(-G // 2, G // 2) if (a * a + b * b + c * c) > (0.25 * G) ** 2)
    assert abs(frac[4] - n_high / (G ** 3 - 1)) < 0.03
    np.testing.assert_array_equal(oracle.mask_from_fraction(frac, 0.85), [1, 0, 0, 1, 0, 0])


def test_channel_mask_keeps_a_smooth_dense_level_and_drops_a_hashed_noise_level():
    """Level 0 (dense, N = 4) holds a linear function of the vertex coordinates, so
    its features vary smoothly; level 1 (hashed, N = 512) holds independent random
    entries, which a 32^3 grid samples as white noise."""
    cfg = S.FieldConfig(n_levels=2, n_feat=2, log2_T=10, base_res=4, max_res=512, norm=S.NORM_LN,
                        hidden_layers=1, width=32)
    flat = S.init_params(cfg, 0).astype(np.float64)
    T = cfg.T
    tab = np.zeros((2, T, 2))
    for zz in range(5):
        for yy in range(5):
            for xx in range(5):
                tab[0, xx + 5 * yy + 25 * zz] = [0.3 * xx - 0.1 * zz, 0.2 * yy]
    tab[1] = np.random.default_rng(1).normal(size=(T, 2))
    flat[: 2 * T * 2] = tab.ravel()
    mask, frac = oracle.channel_mask(flat, cfg, G=32, cutoff=0.25, threshold=0.85)
    np.testing.assert_array_equal(mask, [1, 1, 0, 0])
    assert frac[:2].max() < 0.1 and frac[2:].min() > 0.85


# ---------------------------------------------------------------- 3-D SSIM (Sec. 3.2; Wang et al. 2004)
def test_ssim_of_identical_and_of_constant_volumes():
    """Identical volumes score 1 at every window. For constants a and b every window
    has zero variance and covariance, so the contrast-structure factor is C2 / C2
    and the index is the luminance term (2ab + C1) / (a^2 + b^2 + C1), C1 = 1e-4
    at data range 1. The index is symmetric in its two volumes."""
    rng = np.random.default_rng(3)
    x = rng.random((14, 14, 14))
    y = np.clip(x + 0.2 * rng.standard_normal(x.shape), 0.0, 1.0)
    np.testing.assert_allclose(oracle.ssim_map(x, x), 1.0, rtol=0, atol=1e-13)
    np.testing.assert_allclose(oracle.ssim_map(x, y), oracle.ssim_map(y, x), rtol=0, atol=1e-15)
    for a, b in ((0.0, 0.0), (0.3, 0.7), (1.0, 0.02), (0.5, 0.5)):
        m = oracle.ssim_map(np.full((12, 12, 12), a), np.full((12, 12, 12), b))
        assert m.shape == (2, 2, 2)
        np.testing.assert_allclose(m, (2 * a * b + 1e-4) / (a * a + b * b + 1e-4), rtol=1e-12, atol=0)
    # a data range of 2 scales both constants by 4
    m = oracle.ssim_map(np.full((11, 11, 11), 0.3), np.full((11, 11, 11), 0.9), data_range=2.0)
    np.testing.assert_allclose(m, (2 * 0.27 + 4e-4) / (0.09 + 0.81 + 4e-4), rtol=1e-12, atol=0)


def test_ssim_matches_brute_force_window_and_a_library_filter():
    """One window (D = 11) summed voxel by voxel with the Gaussian written out, and
    a larger volume whose window statistics come from scipy's separable 1-D filter
    along each axis, with variances from E[x^2] - E[x]^2: both equal the oracle's
    direct window sums."""
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(4)
    x = rng.random((11, 11, 11))
    y = 0.5 * x + 0.5 * rng.random((11, 11, 11))
    wsum, sx, sy, sxx, syy, sxy = 0.0, 0.0, 0.0, 0.0, 0.0, 0.0
    for k in range(11):
        for j in range(11):
            for i in range(11):
                w = math.exp(-((i - 5) ** 2 + (j - 5) ** 2 + (k - 5) ** 2) / 4.5)
                a, b = x[k, j, i], y[k, j, i]
                wsum += w
                sx, sy, sxx, syy, sxy = sx + w * a, sy + w * b, sxx + w * a * a, syy + w * b * b, sxy + w * a * b
    mx, my = sx / wsum, sy / wsum
    vx, vy, cxy = sxx / wsum - mx * mx, syy / wsum - my * my, sxy / wsum - mx * my
    c1, c2 = 0.01 ** 2, 0.03 ** 2
    brute = (2 * mx * my + c1) * (2 * cxy + c2) / ((mx * mx + my * my + c1) * (vx + vy + c2))
    got = oracle.ssim_map(x, y)
    assert got.shape == (1, 1, 1)
    assert abs(got[0, 0, 0] - brute) < 1e-12

    D = 23
    x = rng.random((D, D, D))
    y = np.clip(0.8 * x + 0.1 + 0.1 * rng.standard_normal((D, D, D)), 0.0, 1.0)
    g = np.exp(-np.arange(-5, 6) ** 2 / 4.5)
    g /= g.sum()

    def smooth(v):
        for axis in range(3):
            v = ndimage.correlate1d(v, g, axis=axis, mode="constant")
        return v[5:-5, 5:-5, 5:-5]
    mx, my = smooth(x), smooth(y)
    vx, vy, cxy = smooth(x * x) - mx * mx, smooth(y * y) - my * my, smooth(x * y) - mx * my
    lib = (2 * mx * my + c1) * (2 * cxy + c2) / ((mx * mx + my * my + c1) * (vx + vy + c2))
    np.testing.assert_allclose(oracle.ssim_map(x, y), lib, rtol=0, atol=1e-12)


def test_ssim_falls_with_noise_and_vanishes_for_independent_volumes():
    """More additive noise on a smooth volume gives a strictly lower score; two
    independent uniform volumes share no structure, so the covariance term, and
    with it the score, is near 0 (C2 / (2 var + C2) ~ 0.005 per window)."""
    D = 24
    z, y, x = np.meshgrid(*(np.arange(D) / D,) * 3, indexing="ij")
    smooth = 0.5 + 0.4 * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y) * np.sin(np.pi * z)
    noise = np.random.default_rng(5).standard_normal((D, D, D))
    scores = [oracle.ssim(smooth, smooth + s * noise) for s in (0.0, 0.01, 0.03, 0.1, 0.3)]
    assert scores[0] == pytest.approx(1.0, abs=1e-13)
    assert all(a > b for a, b in zip(scores, scores[1:]))
    rng = np.random.default_rng(6)
    assert abs(oracle.ssim(rng.random((D, D, D)), rng.random((D, D, D)))) < 0.05


# ---------------------------------------------------------------- stratified jitter
def test_splitmix64_reference_outputs_and_jittered_strata():
    """SplitMix64 started at 1234567 gives the generator's published first outputs;
    jittered samples stay inside their strata, are uniform there, and seed 0 is the
    midpoint rule."""
    out = oracle.splitmix64(1234567, np.arange(1, 6, dtype=np.uint64))
    assert out.tolist() == [6457827717110365317, 3203168211198807973, 9817491932198370423,
                            4593380528125082431, 16408922859458223821]
    pix = np.arange(0, 4000, 7, dtype=np.int32)
    u = oracle.stratum_offsets(99, pix, 64)
    assert u.dtype == np.float32 and u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.01 and abs(u.var() - 1 / 12) < 0.005
    assert np.array_equal(u[3], oracle.stratum_offsets(99, pix[3:4], 64)[0])     # keyed by pixel
    assert not np.array_equal(u, oracle.stratum_offsets(100, pix, 64))
    assert np.all(oracle.stratum_offsets(0, pix, 64) == np.float32(0.5))
    g = S.GeometryConfig(n_views=3, det_nu=16, det_nv=16)
    tab, du, dv, nu, nv = _geom(g)
    p16 = np.arange(nu * nv)
    o, d, near, far, hit = oracle.ray_setup(tab, du, dv, nu, nv, 1, p16)
    xm, delta = oracle.sample_points(o, d, near, far, 9)
    xj, delta_j = oracle.sample_points(o, d, near, far, 9, oracle.stratum_offsets(5, p16, 9))
    assert np.array_equal(delta, delta_j)
    for r in np.nonzero(hit)[0]:
        # distance of each jittered sample from the entry point, in units of Delta
        s = np.linalg.norm(xj[r].astype(np.float64) - (o[r] + near[r] * d[r]).astype(np.float64), axis=1) / delta[r]
        assert np.all(s > np.arange(9) - 1e-3) and np.all(s < np.arange(9) + 1 + 1e-3)


# ---------------------------------------------------------------- measurement model
def test_poisson_measurement_has_the_poisson_moments_and_the_count_floor():
    """Measured projections (Sec. 3.1; the measurement model of the benchmark
    workloads): I ~ Poisson(I0 exp(-A)), A_meas = -ln(max(I, 1) / I0). The counts
    recovered from A_meas must have the Poisson mean and variance lambda = I0 e^-A
    (each within 5 standard errors over 200 000 draws), A_meas must centre on A
    (delta method: bias ~ 1/(2 lambda), spread ~ 1/sqrt(lambda)), and where lambda
    is far below one count the floor max(I, 1) caps A_meas at ln I0."""
    I0, n = 1e5, 200_000
    for A, seed in ((0.0, 1), (0.5, 2), (1.7, 3), (4.0, 4), (7.0, 5)):
        lam = I0 * math.exp(-A)
        am = S.poisson_measure(np.full(n, A), I0, seed)
        assert am.dtype == np.float32 and am.shape == (n,)
        counts = np.rint(I0 * np.exp(-am.astype(np.float64)))
        se_mean = math.sqrt(lam / n)
        se_var = math.sqrt((lam + 2.0 * lam * lam) / n)
        assert abs(counts.mean() - lam) < 5.0 * se_mean, (A, counts.mean(), lam)
        assert abs(counts.var() - lam) < 5.0 * se_var, (A, counts.var(), lam)
        assert abs(float(am.astype(np.float64).mean()) - A) < 1.0 / lam + 5.0 / math.sqrt(lam * n), A
    # lambda = I0 e^-25 ~ 1.4e-6: nearly every draw counts zero, floored to one count.
    am = S.poisson_measure(np.full(10_000, 25.0), I0, 6)
    assert np.all(np.isfinite(am))
    assert float(am.max()) == float(np.float32(math.log(I0)))
    assert np.mean(am == np.float32(math.log(I0))) > 0.999
    # Seeded: the same seed repeats the draw, another seed does not.
    a = np.linspace(0.0, 2.0, 1000)
    assert np.array_equal(S.poisson_measure(a, I0, 9), S.poisson_measure(a, I0, 9))
    assert not np.array_equal(S.poisson_measure(a, I0, 9), S.poisson_measure(a, I0, 10))


# ---------------------------------------------------------------- stored record
def test_oracle_reproduces_its_stored_step():
    """tests/golden/oracle_step.json (written by tests/golden/make_golden.py from the
    oracle alone) still matches the oracle: a change to the oracle's arithmetic shows
    up here and must be justified and the record rewritten."""
    import json
    import os
    import sys
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    sys.path.insert(0, here)
    import make_golden
    ref = json.load(open(os.path.join(here, "oracle_step.json")))
    now = make_golden.expected()
    assert now["pix"] == ref["pix"] and now["grad_index"] == ref["grad_index"]
    np.testing.assert_allclose(now["A"], ref["A"], rtol=1e-12, atol=0)
    assert abs(now["loss"] - ref["loss"]) <= 1e-12 * ref["loss"]
    np.testing.assert_allclose(now["grad_value"], ref["grad_value"], rtol=1e-10, atol=1e-15)
    np.testing.assert_allclose(now["param_after_adam"], ref["param_after_adam"], rtol=1e-12, atol=0)
