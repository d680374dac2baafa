"""CUDA path vs the CPU oracle, element by element, through the C ABI.

Tolerances (from the method's arithmetic and the stated targets): sample
positions, deltas and corner indices bitwise; features and per-point mu 1e-5
relative (float32 accumulation of <= 8 L terms and a 5-layer MLP); ray sums and
losses 1e-5 relative; gradients 1e-3 relative (float32 accumulation in a
different order, scatter atomics reorder sums).
"""
import math

import numpy as np
import pytest

import oracle
import synthetic as S
from _cases import (C4_SUB, C4_SUB_GEOM, C4_SUB_N, batch, c4_subinstance, field_cfg, fp32_gradient_errors,
                    kink_free_rays,
                    hit_pixels, oracle_geom, replace, rounded_tables)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _t(a, dtype=None):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _np(t):
    return t.detach().cpu().numpy()


GEOM = S.GeometryConfig(n_views=6, det_nu=40, det_nv=36)


def _group_errors(g_gpu, g_orc, cfg):
    """Per parameter group: (max |error| / max |ref|, ||error|| / ||ref||)."""
    lay = S.param_layout(cfg)
    out = {}
    for name in ("tables", "gamma", "beta") + tuple(f"{p}{k}" for k in range(cfg.hidden_layers + 1)
                                                 for p in ("W", "b")):
        o, n = lay[name]
        a, b = g_gpu[o:o + n].astype(np.float64), g_orc[o:o + n]
        scale = np.abs(b).max()
        if scale == 0:
            out[name] = (0.0 if np.abs(a).max() == 0 else np.inf, 0.0)
            continue
        d = a - b
        out[name] = (np.abs(d).max() / scale, np.linalg.norm(d) / np.linalg.norm(b))
    return out


def _grad_close(g_gpu, g_orc, cfg, rtol=1e-3, what="", norm_rtol=None):
    """Every group within rtol of its largest entry (max-abs); with norm_rtol, the
    group's error norm is bounded relative to the gradient norm instead."""
    errs = _group_errors(g_gpu, g_orc, cfg)
    print(what, {k: (f"{v[0]:.2e}", f"{v[1]:.2e}") for k, v in errs.items()})
    bad = {k: v for k, v in errs.items() if (v[1] > norm_rtol if norm_rtol is not None else v[0] > rtol)}
    assert not bad, (what, bad)


# ------------------------------------------------------------------------------ stages
@pytest.mark.parametrize("jitter", [0, 0x5EED0123456789AB])
@pytest.mark.parametrize("N", [1, 37, 64, 200])
def test_sampler_positions_and_deltas_are_bitwise(lib, N, jitter):
    geom = lib.Geometry.from_config(GEOM)
    tab, du, dv = geom.view_table()
    otab, odu, odv, nu, nv = oracle_geom(GEOM)
    assert np.array_equal(tab.view(np.uint32), otab.view(np.uint32))
    assert np.float32(du) == odu and np.float32(dv) == odv
    pix = np.arange(nu * nv, dtype=np.int32)          # every pixel, hits and misses
    for view in (0, 2, 5):
        xyz = torch.empty(len(pix) * N * 3, device="cuda")
        delta = torch.empty(len(pix), device="cuda")
        lib.sample_rays(geom, view, _t(pix), N, xyz, delta, jitter_seed=jitter)
        o, d, near, far, hit = oracle.ray_setup(otab, odu, odv, nu, nv, view, pix)
        u = oracle.stratum_offsets(jitter, pix, N) if jitter else None
        x, dl = oracle.sample_points(o, d, near, far, N, u)
        g = _np(xyz).reshape(len(pix), N, 3)
        assert np.array_equal(_np(delta).view(np.uint32), dl.view(np.uint32))
        assert np.array_equal(g[hit].view(np.uint32), x[hit].view(np.uint32))


@pytest.mark.parametrize("L,log2T,base,top", [(8, 12, 4, 48), (16, 8, 2, 512), (8, 20, 16, 64)])
def test_corner_indices_are_bitwise(lib, L, log2T, base, top):
    cfg = field_cfg(n_levels=L, log2_T=log2T, base_res=base, max_res=top)
    field = lib.Field(cfg, params=S.init_params(cfg, 0))
    assert field.level_resolutions() == oracle.level_resolutions(L, base, top)
    rng = np.random.default_rng(L + log2T)
    pts = rng.random((3000, 3)).astype(np.float32)
    pts[:8] = [[0, 0, 0], [1, 1, 1], [1, 0, 0.5], [0.5, 0.5, 0.5], [-0.1, 0.3, 1.2],
               [np.float32(1) - np.float32(2 ** -24), 0.25, 0.75], [0.125, 0.5, 0.875], [1e-30, 0.9999, 0.5]]
    idx = torch.empty(len(pts) * L * 8, dtype=torch.int32, device="cuda")
    w = torch.empty(len(pts) * L * 8, device="cuda")
    lib.hash_corners(field, _t(pts), idx, w)
    oi, ow, _ = oracle.corners(pts, oracle.level_resolutions(L, base, top), 1 << log2T)
    assert np.array_equal(_np(idx).view(np.uint32).reshape(oi.shape), oi)
    np.testing.assert_allclose(_np(w).reshape(ow.shape), ow, rtol=0, atol=2e-7)


@pytest.mark.parametrize("precision", [S.PREC_F32, S.PREC_BF16, S.PREC_F16])
def test_gather_features_match_oracle(lib, precision):
    cfg = field_cfg(n_levels=16, log2_T=10, base_res=3, max_res=300, precision=precision)
    flat = S.init_params(cfg, 1, table_scale=1.0)
    field = lib.Field(cfg, params=flat)
    pts = np.random.default_rng(5).random((4097, 3)).astype(np.float32)
    h = torch.empty(len(pts) * cfg.d_in, device="cuda")
    lib.encode_points(field, _t(pts), h)
    ref_flat = rounded_tables(flat, cfg, precision)
    tables = oracle.unflatten(ref_flat.astype(np.float64), cfg)["tables"]
    ref = oracle.encode(pts, tables, oracle.level_resolutions(16, 3, 300), cfg.T)
    np.testing.assert_allclose(_np(h).reshape(ref.shape), ref, rtol=0, atol=1e-5 * np.abs(ref).max())


@pytest.mark.parametrize("precision", [S.PREC_F32, S.PREC_BF16])
@pytest.mark.parametrize("ordered", [False, True])
def test_scatter_stage_matches_oracle(lib, precision, ordered):
    """The scatter stage alone (warp-segmented runs and direct atomics): the float32
    gradient tables equal the oracle's scatter-add within 1e-5 of their largest entry,
    for random points and for points in ray order (long runs of one cell at coarse
    levels), 4099 points (a ragged last warp)."""
    cfg = field_cfg(n_levels=16, log2_T=10, base_res=3, max_res=300, precision=precision)
    field = lib.Field(cfg, params=S.init_params(cfg, 2))
    rng = np.random.default_rng(6)
    n = 4099
    if ordered:
        t = np.linspace(0.0, 1.0, n)[:, None]
        pts = (0.1 + 0.8 * t * np.array([[0.9, 0.7, 0.3]])).astype(np.float32)
    else:
        pts = rng.random((n, 3)).astype(np.float32)
    dh = rng.normal(size=(n, cfg.d_in)).astype(np.float32)
    field.grads.zero_()
    lib.scatter_points(field, _t(pts), _t(dh))
    res = oracle.level_resolutions(16, 3, 300)
    ref = oracle.encode_backward(pts, dh.astype(np.float64), res, cfg.T, cfg.n_feat).ravel()
    g = _np(field.flat_grads())[:ref.size]
    assert np.abs(g - ref).max() <= 1e-5 * np.abs(ref).max()
    assert float(field.grads[ref.size:].abs().max()) == 0.0


def test_roofline_probes_run_and_count(lib):
    buf = torch.zeros(1 << 20, device="cuda")
    sink = torch.zeros(1, device="cuda")
    lib.probe_l2_read(buf, 3, sink)
    assert lib.probe_random_gather(buf, 8, 100000, sink) >= 100000
    assert lib.probe_random_gather(buf, 4, 1000, sink) >= 1000
    red = torch.zeros(1 << 12, device="cuda")
    n = lib.probe_random_red(red, 50000)
    torch.cuda.synchronize()
    assert n >= 50000 and float(red.sum()) == pytest.approx(n * 2 * 1e-30, rel=1e-3)
    assert float(sink[0]) == 0.0


# ------------------------------------------------------------------------------ forward
FWD_CASES = [
    dict(norm=S.NORM_LN, n_levels=16, hidden_layers=4, log2_T=12, max_res=200),
    dict(norm=S.NORM_LN_PER_LEVEL, n_levels=8, hidden_layers=2),
    dict(norm=S.NORM_NONE, n_levels=8, hidden_layers=1, log2_T=8),
    dict(norm=S.NORM_LN, n_levels=16, hidden_layers=3, log2_T=16, max_res=1024),
]


@pytest.mark.parametrize("case", range(len(FWD_CASES)))
@pytest.mark.parametrize("N", [45, 64])
def test_render_forward_matches_oracle(lib, case, N):
    cfg = field_cfg(**FWD_CASES[case])
    flat = S.init_params(cfg, 10 + case, table_scale=0.5)
    field = lib.Field(cfg, params=flat)
    mask = np.ones(cfg.d_in, dtype=np.float32)
    mask[3] = 0.0
    field.set_channel_mask(mask)
    geom = lib.Geometry.from_config(GEOM)
    pix = batch(GEOM, 4, 300, seed=case, n_miss=5)
    ws = lib.workspace(lib.step_workspace_bytes(field, len(pix), N))
    a = torch.empty(len(pix), device="cuda")
    lib.render_forward(field, geom, 4, _t(pix), N, a, ws)
    ref = oracle.render(flat.astype(np.float64), cfg, oracle_geom(GEOM), 4, pix, N, mask)
    np.testing.assert_allclose(_np(a), ref, rtol=1e-5, atol=1e-6)
    assert np.all(_np(a)[-5:] == 0.0)          # rays that miss the volume


# ------------------------------------------------------------------------------ backward
@pytest.mark.parametrize("case", range(len(FWD_CASES)))
@pytest.mark.parametrize("loss", [S.LOSS_MSE, S.LOSS_L1])
def test_train_step_loss_and_gradients_match_oracle(lib, case, loss):
    cfg = field_cfg(**FWD_CASES[case], loss=loss)
    flat = S.init_params(cfg, 20 + case, table_scale=0.5).astype(np.float32)
    N = 53
    geom = lib.Geometry.from_config(GEOM)
    og = oracle_geom(GEOM)
    pix = batch(GEOM, 1, 257, seed=case + 7, n_miss=3)
    a_meas = np.random.default_rng(case).uniform(0, 0.8, size=len(pix)).astype(np.float32)
    A, cache = oracle.render_forward(flat.astype(np.float64), cfg, og, 1, pix, N)
    ref_loss, dLdA = oracle.loss_and_grad(A, a_meas, loss)
    ref_grad = oracle.render_backward(cache, dLdA, cfg)

    field = lib.Field(cfg, params=flat)
    ws = lib.workspace(lib.step_workspace_bytes(field, len(pix), N))
    # gradient through render_backward with the oracle's dL/dA
    lib.render_backward(field, geom, 1, _t(pix), N, _t(dLdA.astype(np.float32)), ws)
    g = _np(field.flat_grads())
    _grad_close(g, ref_grad, cfg, what="render_backward")
    field.grads.zero_()
    # the full step: loss, then Adam applied (grads zeroed afterwards)
    loss_t = torch.zeros(1, device="cuda")
    lib.train_step(field, geom, 1, _t(pix), _t(a_meas), N, loss_t, ws)
    assert abs(_np(loss_t)[0] - ref_loss) <= 1e-5 * abs(ref_loss)
    assert float(field.grads.abs().max()) == 0.0
    flags, scale, step = field.poll_status()
    assert step == 1 and flags == 0


@pytest.mark.parametrize("precision", [S.PREC_F32, S.PREC_BF16])
@pytest.mark.parametrize("N", [64, 80, 150, 192, 300, 512, 520])
def test_train_step_fused_and_split_paths_match_oracle(lib, precision, N):
    """accumulate_step runs one fused forward+loss+backward kernel when a ray has at
    most 16 chunks of 32 samples (N <= 512: several rays per CTA up to 8 chunks, one
    ray per CTA for N = 300 and the largest fused ray, N = 512) and separate kernels
    otherwise (N = 520). N = 80 (two rays of 3 chunks per 6-warp CTA), 150 (one ray
    of 5 chunks) and 192 (6 chunks) take the 16-bit path's CTA-cooperative weight
    gradient, with rays that miss the volume in the batch. Each gives the oracle's loss (FP32 within 1e-5) and every
    gradient group element by element (FP32 within 1e-3 of the group's largest
    entry, BF16 within the mixed norm bound); train_step then gives the same loss,
    applies Adam and zeroes the gradients."""
    cfg = field_cfg(n_levels=16, hidden_layers=4, log2_T=12, max_res=256, precision=precision,
                    loss_scale_init=1.0)
    flat = S.init_params(cfg, 40, table_scale=0.5).astype(np.float32)
    field = lib.Field(cfg, params=flat)
    geom = lib.Geometry.from_config(GEOM)
    og = oracle_geom(GEOM)
    pix = batch(GEOM, 2, 190, seed=N, n_miss=2)
    a_meas = np.random.default_rng(N).uniform(0, 0.8, size=len(pix)).astype(np.float32)
    ref_flat = rounded_tables(flat, cfg, precision).astype(np.float64)
    A, cache = oracle.render_forward(ref_flat, cfg, og, 2, pix, N)
    ref_loss, dLdA = oracle.loss_and_grad(A, a_meas, S.LOSS_MSE)
    g_ref = oracle.render_backward(cache, dLdA, cfg)
    ws = lib.workspace(lib.step_workspace_bytes(field, len(pix), N))
    tol_f = 1e-5 if precision == S.PREC_F32 else 2 * MIXED_TOL[precision][0]
    loss_t = torch.zeros(1, device="cuda")
    lib.accumulate_step(field, geom, 2, _t(pix), _t(a_meas), N, loss_t, ws)
    assert abs(_np(loss_t)[0] - ref_loss) <= tol_f * ref_loss
    g = _np(field.flat_grads())
    if precision == S.PREC_F32:
        bad = fp32_gradient_errors(g, g_ref, cfg, cache, dLdA)
        assert not bad, (f"fused/split N={N}", bad)
    else:
        _grad_close(g, g_ref, cfg, what=f"fused/split N={N}", norm_rtol=MIXED_TOL[precision][1])
    field.grads.zero_()
    loss_t.zero_()
    lib.train_step(field, geom, 2, _t(pix), _t(a_meas), N, loss_t, ws)
    assert abs(_np(loss_t)[0] - ref_loss) <= tol_f * ref_loss
    assert float(field.grads.abs().max()) == 0.0
    flags, _, step = field.poll_status()
    assert step == 1 and flags == 0
    assert not np.array_equal(_np(field.flat_params()), flat)


@pytest.mark.parametrize("hidden", [6, 8])
def test_deep_mlp_with_long_rays_takes_the_split_kernels(lib, hidden):
    """A fused CTA keeps 32 H tensor-memory columns a thread for every group of four
    warps. With 6 or 8 hidden layers and rays of 10 chunks (N = 300) that exceeds the
    SM's 512 columns, so accumulate_step declines the fused kernel before launching
    anything and runs forward, loss and backward as separate kernels; the loss and
    every gradient group still match the oracle (FP32 bounds). Rays with a sample
    at a ReLU kink (within float32 rounding, where either branch is correct) are
    left out of the batch, so that every group has one correct gradient; deep
    random-init MLPs put a few such units in the first layers."""
    N = 300
    cfg = field_cfg(n_levels=16, hidden_layers=hidden, log2_T=12, max_res=256, loss_scale_init=1.0)
    flat = S.init_params(cfg, 41, table_scale=0.5).astype(np.float32)
    field = lib.Field(cfg, params=flat)
    geom = lib.Geometry.from_config(GEOM)
    og = oracle_geom(GEOM)
    pix = batch(GEOM, 3, 120, seed=hidden, n_miss=2)
    _, cache = oracle.render_forward(flat.astype(np.float64), cfg, og, 3, pix, N)
    pix = pix[kink_free_rays(cache, len(pix))]
    assert len(pix) >= 80
    a_meas = np.random.default_rng(hidden).uniform(0, 0.8, size=len(pix)).astype(np.float32)
    A, cache = oracle.render_forward(flat.astype(np.float64), cfg, og, 3, pix, N)
    ref_loss, dLdA = oracle.loss_and_grad(A, a_meas, S.LOSS_MSE)
    g_ref = oracle.render_backward(cache, dLdA, cfg)
    ws = lib.workspace(lib.step_workspace_bytes(field, len(pix), N))
    loss_t = torch.zeros(1, device="cuda")
    lib.accumulate_step(field, geom, 3, _t(pix), _t(a_meas), N, loss_t, ws)
    assert abs(_np(loss_t)[0] - ref_loss) <= 1e-5 * ref_loss
    bad = fp32_gradient_errors(_np(field.flat_grads()), g_ref, cfg, cache, dLdA)
    assert not bad, (f"H={hidden} N={N}", bad)


@pytest.mark.parametrize("N", [192, 520])
def test_stratified_jitter_training_matches_oracle(lib, N):
    """Stratified jitter (a new SplitMix64 seed per step): the fused (N = 192) and the
    split (N = 520) paths give the oracle's loss for the same jittered samples, and
    render_backward the oracle's gradient."""
    cfg = field_cfg(n_levels=16, hidden_layers=4, log2_T=12, max_res=256)
    flat = S.init_params(cfg, 41, table_scale=0.5).astype(np.float32)
    field = lib.Field(cfg, params=flat)
    geom = lib.Geometry.from_config(GEOM)
    og = oracle_geom(GEOM)
    pix = batch(GEOM, 4, 150, seed=N, n_miss=2)
    a_meas = np.random.default_rng(N + 1).uniform(0, 0.8, size=len(pix)).astype(np.float32)
    seed = 0xC0FFEE + N
    A, cache = oracle.render_forward(flat.astype(np.float64), cfg, og, 4, pix, N, jitter_seed=seed)
    A_mid = oracle.render(flat.astype(np.float64), cfg, og, 4, pix, N)
    assert np.abs(A - A_mid).max() > 1e-6            # the jitter moves the samples
    ref_loss, dLdA = oracle.loss_and_grad(A, a_meas, S.LOSS_MSE)
    ws = lib.workspace(lib.step_workspace_bytes(field, len(pix), N))
    lib.render_backward(field, geom, 4, _t(pix), N, _t(dLdA.astype(np.float32)), ws, jitter_seed=seed)
    _grad_close(_np(field.flat_grads()), oracle.render_backward(cache, dLdA, cfg), cfg, what="jitter")
    field.grads.zero_()
    loss_t = torch.zeros(1, device="cuda")
    lib.accumulate_step(field, geom, 4, _t(pix), _t(a_meas), N, loss_t, ws, jitter_seed=seed)
    assert abs(_np(loss_t)[0] - ref_loss) <= 1e-5 * ref_loss


def test_autograd_function_matches_oracle(lib):
    cfg = field_cfg(n_levels=16, hidden_layers=4, log2_T=10, max_res=300)
    flat = S.init_params(cfg, 3, table_scale=0.5).astype(np.float32)
    field = lib.Field(cfg, params=flat)
    geom = lib.Geometry.from_config(GEOM)
    pix = batch(GEOM, 2, 128, seed=9)
    p = field.flat_params().clone().requires_grad_(True)
    a = lib.Render.apply(p, field, geom, 2, _t(pix), 40)
    a_meas = _t(np.full(len(pix), 0.3, dtype=np.float32))
    loss = ((a - a_meas) ** 2).mean()
    loss.backward()
    A, cache = oracle.render_forward(flat.astype(np.float64), cfg, oracle_geom(GEOM), 2, pix, 40)
    _, dLdA = oracle.loss_and_grad(A, np.full(len(pix), 0.3), S.LOSS_MSE)
    _grad_close(_np(p.grad), oracle.render_backward(cache, dLdA, cfg), cfg, what="autograd")


# Mixed precision: the MLP runs on tensor cores with 16-bit inputs, weights and
# activations (float32 accumulation), u = 2^-9 (bf16) or 2^-12 (f16) per rounding.
# Forward: the error compounds over the 5 layers to a few u relative on mu and A
# (bound: 15 u for bf16, 25 u for f16, relative to the largest A). Gradients: the
# dominant term is ReLU masks that flip where a pre-activation lies within rounding
# distance of zero; the number of flips grows like u and each costs an O(1) term, so
# the error norm of a parameter group grows like sqrt(u) (measured: bf16 3-6%, f16
# 1-2%, about sqrt(u) = 4.4% / 1.6%). Bound: 2 sqrt(u) of the group's gradient
# norm. A layout mistake (a transposed weight, a wrong fragment row) costs O(1).
MIXED_TOL = {S.PREC_BF16: (15 * 2.0 ** -9, 2 * 2.0 ** -4.5),
             S.PREC_F16: (25 * 2.0 ** -12, 2 * 2.0 ** -6)}   # (forward, gradient norm)


def _scale(precision):
    """FP16 backward values (~1e-6) are subnormal without a loss scale."""
    return 1024.0 if precision == S.PREC_F16 else 1.0


@pytest.mark.parametrize("precision", [S.PREC_BF16, S.PREC_F16])
@pytest.mark.parametrize("case", [0, 1, 2])
def test_mixed_precision_forward_and_gradients_track_oracle(lib, precision, case):
    cfg = field_cfg(**FWD_CASES[case], precision=precision, loss_scale_init=_scale(precision))
    flat = S.init_params(cfg, 30 + case, table_scale=0.5).astype(np.float32)
    field = lib.Field(cfg, params=flat)
    geom = lib.Geometry.from_config(GEOM)
    og = oracle_geom(GEOM)
    N = 61
    pix = batch(GEOM, 3, 200, seed=case, n_miss=2)
    ref_flat = rounded_tables(flat, cfg, precision).astype(np.float64)
    ws = lib.workspace(lib.step_workspace_bytes(field, len(pix), N))
    a = torch.empty(len(pix), device="cuda")
    lib.render_forward(field, geom, 3, _t(pix), N, a, ws)
    A, cache = oracle.render_forward(ref_flat, cfg, og, 3, pix, N)
    tol_f, tol_g = MIXED_TOL[precision]
    err = np.abs(_np(a) - A).max() / np.abs(A).max()
    assert err <= tol_f, err
    a_meas = np.random.default_rng(case).uniform(0, 0.8, size=len(pix)).astype(np.float32)
    _, dLdA = oracle.loss_and_grad(A, a_meas, S.LOSS_MSE)
    lib.render_backward(field, geom, 3, _t(pix), N, _t(dLdA.astype(np.float32)), ws)
    g = _np(field.flat_grads()) / cfg.loss_scale_init
    _grad_close(g, oracle.render_backward(cache, dLdA, cfg), cfg, what=f"mixed {precision}", norm_rtol=tol_g)


@pytest.mark.parametrize("precision", [S.PREC_F32, S.PREC_BF16])
def test_c4_subinstance_gradients_match_oracle(lib, precision):
    """The large configuration's field shape (L16, 16..2048, T = 2^8 with forced
    collisions, 4x32 MLP) on the seeded 16^3 sub-instance whose oracle gradient is
    pinned by central differences: the library's backward gives the oracle gradient
    (FP32 within 1e-3 of each group's largest entry; BF16 within the mixed-precision
    norm bound) and the oracle loss."""
    cfg = replace(C4_SUB, precision=precision)
    og, flat64, pix, A_meas = c4_subinstance()
    flat = flat64.astype(np.float32)
    ref_flat = rounded_tables(flat, cfg, precision).astype(np.float64)
    A, cache = oracle.render_forward(ref_flat, cfg, og, 1, pix, C4_SUB_N)
    ref_loss, dLdA = oracle.loss_and_grad(A, A_meas, S.LOSS_MSE)
    ref_grad = oracle.render_backward(cache, dLdA, cfg)
    field = lib.Field(cfg, params=flat)
    geom = lib.Geometry.from_config(C4_SUB_GEOM)
    ws = lib.workspace(lib.step_workspace_bytes(field, len(pix), C4_SUB_N))
    lib.render_backward(field, geom, 1, _t(pix), C4_SUB_N, _t(dLdA.astype(np.float32)), ws)
    g = _np(field.flat_grads())
    if precision == S.PREC_F32:
        _grad_close(g, ref_grad, cfg, what="c4 sub f32")
    else:
        _grad_close(g, ref_grad, cfg, what="c4 sub bf16", norm_rtol=MIXED_TOL[precision][1])
    field.grads.zero_()
    loss_t = torch.zeros(1, device="cuda")
    lib.accumulate_step(field, geom, 1, _t(pix), _t(A_meas.astype(np.float32)), C4_SUB_N, loss_t, ws)
    tol = 1e-5 if precision == S.PREC_F32 else 2 * MIXED_TOL[precision][0]
    assert abs(_np(loss_t)[0] - ref_loss) <= tol * ref_loss


@pytest.mark.parametrize("precision", [S.PREC_BF16, S.PREC_F16])
def test_mixed_precision_voxel_loss_and_query(lib, precision):
    cfg = field_cfg(n_levels=16, hidden_layers=4, log2_T=12, max_res=256, precision=precision,
                    loss_scale_init=_scale(precision))
    flat = S.init_params(cfg, 16, table_scale=0.5).astype(np.float32)
    field = lib.Field(cfg, params=flat)
    ref_flat = rounded_tables(flat, cfg, precision).astype(np.float64)
    tol_f, tol_g = MIXED_TOL[precision]
    rng = np.random.default_rng(4)
    xyz = rng.random((1001, 3)).astype(np.float32)
    mu = torch.empty(1001, device="cuda")
    lib.query_points(field, _t(xyz), mu)
    ref_mu = oracle.query_points(ref_flat, cfg, xyz)
    assert np.abs(_np(mu) - ref_mu).max() <= tol_f
    D = 9
    vol = torch.empty(D ** 3, device="cuda")
    lib.query_volume(field, D, vol)
    assert np.abs(_np(vol).reshape(D, D, D) - oracle.query_volume(ref_flat, cfg, D)).max() <= tol_f
    # targets 0.15..0.3 away from mu: sign(mu - mu_gt) must not hinge on rounding
    off = rng.uniform(0.15, 0.3, size=1001)
    mu_gt = np.where(ref_mu > 0.5, ref_mu - off, ref_mu + off).astype(np.float32)
    ws = lib.workspace(lib.points_workspace_bytes(field, 1001))
    loss_t = torch.zeros(1, device="cuda")
    lib.fit_points_backward(field, _t(xyz), _t(mu_gt), loss_t, ws)
    st = oracle.AdamState.zeros(flat.size)
    _, _, ref_loss, ref_grad = oracle.fit_points_step(ref_flat, st, cfg, xyz, mu_gt, adam=False)
    assert abs(_np(loss_t)[0] - ref_loss) <= tol_f * ref_loss
    g = _np(field.flat_grads()) / cfg.loss_scale_init
    _grad_close(g, ref_grad, cfg, what="mixed voxel loss", norm_rtol=tol_g)


def reachable_params(cfg):
    """Mask of the parameters the optimizer visits: every entry of a hashed level,
    the first (N_l + 1)^3 entries of a dense level (a corner index there is at most
    (N_l + 1)^3 - 1), its float count rounded up to a multiple of four, and the
    LN / MLP block. Every parameter a step can give a gradient is inside."""
    from oracle.encoding import is_dense, level_resolutions
    T, F = 2 ** cfg.log2_T, cfg.n_feat
    n = S.param_layout(cfg)["_total"][1]
    live = np.zeros(n, dtype=bool)
    for l, res in enumerate(level_resolutions(cfg.n_levels, cfg.base_res, cfg.max_res)):
        n_l = (res + 1) ** 3 if is_dense(res, T) else T
        live[l * T * F: l * T * F + min(T * F, -(-n_l * F // 4) * 4)] = True
    live[cfg.n_levels * T * F:] = True
    return live


def test_adam_matches_oracle(lib):
    # gradients on every parameter a step can reach (this field has dense levels
    # with unreachable entries, which the next test covers)
    cfg = field_cfg(n_levels=8, log2_T=8)
    flat = S.init_params(cfg, 4).astype(np.float32)
    live = reachable_params(cfg)
    assert not live.all()
    field = lib.Field(cfg, params=flat)
    rng = np.random.default_rng(0)
    st = oracle.AdamState.zeros(flat.size)
    p_ref = flat.astype(np.float64)
    for k in range(3):
        g = (rng.normal(size=flat.size) * rng.choice([0, 1e-6, 1e-2, 1], size=flat.size)).astype(np.float32)
        g[~live] = 0.0
        field.grads[: flat.size].copy_(_t(g))
        lib.optimizer_step(field)
        p_ref, st, _ = oracle.adam_step(p_ref, g.astype(np.float64), st, cfg)
        np.testing.assert_allclose(_np(field.flat_params()), p_ref, rtol=2e-6, atol=2e-8)
        assert float(field.grads.abs().max()) == 0.0


def test_adam_leaves_unreachable_table_entries(lib):
    # Adam visits only the reachable parameters: entries past a dense level's
    # (N_l + 1)^3 vertices keep their values, gradients and moments (a step never
    # gives them a gradient, so for the method this is the dense update exactly)
    cfg = field_cfg(n_levels=8, log2_T=10)
    flat = S.init_params(cfg, 6).astype(np.float32)
    live = reachable_params(cfg)
    dead = ~live
    assert dead.sum() > 100
    field = lib.Field(cfg, params=flat)
    rng = np.random.default_rng(3)
    g = rng.normal(size=flat.size).astype(np.float32)
    field.grads[: flat.size].copy_(_t(g))
    lib.optimizer_step(field)
    st = oracle.AdamState.zeros(flat.size)
    p_ref, st, _ = oracle.adam_step(flat.astype(np.float64), np.where(live, g, 0.0), st, cfg)
    p = _np(field.flat_params())
    np.testing.assert_allclose(p[live], p_ref[live], rtol=2e-6, atol=2e-8)
    np.testing.assert_array_equal(p[dead], flat[dead])
    np.testing.assert_array_equal(_np(field.grads[: flat.size])[dead], g[dead])
    assert float(field.grads[: flat.size][_t(live)].abs().max()) == 0.0
    assert float(field.adam_m[: flat.size][_t(dead)].abs().max()) == 0.0


def test_training_curve_tracks_oracle(lib):
    cfg = field_cfg(n_levels=8, hidden_layers=2, log2_T=12, norm=S.NORM_LN_PER_LEVEL)
    flat = S.init_params(cfg, 5).astype(np.float32)
    field = lib.Field(cfg, params=flat)
    geom = lib.Geometry.from_config(GEOM)
    og = oracle_geom(GEOM)
    vol, _ = S.phantom(S.WORKLOADS["tiny_fp32"], seed=0, D=24)
    proj = oracle.project(og, vol, oversample=1)
    rng = np.random.default_rng(11)
    st = oracle.AdamState.zeros(flat.size)
    p_ref = flat.astype(np.float64)
    N = 32
    loss_t = torch.zeros(1, device="cuda")
    for step in range(6):
        view = int(rng.integers(0, GEOM.n_views))
        pix = rng.choice(hit_pixels(GEOM, view), size=200, replace=False).astype(np.int32)
        a_meas = proj[view].ravel()[pix].astype(np.float32)
        ws = lib.workspace(lib.step_workspace_bytes(field, len(pix), N))
        lib.train_step(field, geom, view, _t(pix), _t(a_meas), N, loss_t, ws)
        p_ref, st, ref_loss, _ = oracle.train_step(p_ref, st, cfg, og, view, pix, a_meas, N)
        assert abs(_np(loss_t)[0] - ref_loss) <= 1e-3 * ref_loss, (step, _np(loss_t)[0], ref_loss)


# ------------------------------------------------------------------------------ points / MCI
@pytest.mark.parametrize("norm", [S.NORM_LN, S.NORM_NONE])
def test_voxel_loss_gradients_match_oracle(lib, norm):
    cfg = field_cfg(n_levels=16, hidden_layers=4, log2_T=12, max_res=256, norm=norm)
    flat = S.init_params(cfg, 6, table_scale=0.5).astype(np.float32)
    field = lib.Field(cfg, params=flat)
    rng = np.random.default_rng(2)
    xyz = rng.random((1000, 3)).astype(np.float32)
    mu_gt = rng.random(1000).astype(np.float32)
    ws = lib.workspace(lib.points_workspace_bytes(field, len(xyz)))
    loss_t = torch.zeros(1, device="cuda")
    lib.fit_points_backward(field, _t(xyz), _t(mu_gt), loss_t, ws)
    st = oracle.AdamState.zeros(flat.size)
    _, _, ref_loss, ref_grad = oracle.fit_points_step(flat.astype(np.float64), st, cfg, xyz, mu_gt, adam=False)
    assert abs(_np(loss_t)[0] - ref_loss) <= 1e-5 * ref_loss
    _grad_close(_np(field.flat_grads()), ref_grad, cfg, what="voxel loss")


def test_query_volume_and_points_match_oracle(lib):
    cfg = field_cfg(n_levels=16, hidden_layers=4, log2_T=12, max_res=256)
    flat = S.init_params(cfg, 7, table_scale=0.5).astype(np.float32)
    field = lib.Field(cfg, params=flat)
    D = 13
    out = torch.empty(D ** 3, device="cuda")
    lib.query_volume(field, D, out)
    ref = oracle.query_volume(flat.astype(np.float64), cfg, D)
    np.testing.assert_allclose(_np(out).reshape(D, D, D), ref, rtol=0, atol=1e-5)
    xyz = np.random.default_rng(1).random((777, 3)).astype(np.float32)
    mu = torch.empty(777, device="cuda")
    lib.query_points(field, _t(xyz), mu)
    np.testing.assert_allclose(_np(mu), oracle.query_points(flat.astype(np.float64), cfg, xyz), rtol=0, atol=1e-5)


def test_projector_matches_oracle(lib):
    g = S.GeometryConfig(n_views=3, det_nu=24, det_nv=20)
    geom = lib.Geometry.from_config(g)
    vol, _ = S.phantom(S.WORKLOADS["tiny_fp32"], seed=3, D=20)
    out = torch.empty(3 * 20 * 24, device="cuda")
    lib.project(geom, _t(vol.astype(np.float32)), 2, out)
    ref = oracle.project(oracle_geom(g), vol.astype(np.float32).astype(np.float64), oversample=2)
    np.testing.assert_allclose(_np(out).reshape(ref.shape), ref, rtol=1e-5, atol=1e-6)


# ------------------------------------------------------------------------------ edge cases
def test_empty_batch_and_all_miss(lib):
    cfg = field_cfg()
    flat = S.init_params(cfg, 8).astype(np.float32)
    field = lib.Field(cfg, params=flat)
    geom = lib.Geometry.from_config(GEOM)
    ws = lib.workspace(lib.step_workspace_bytes(field, 0, 16))
    loss_t = torch.full((1,), 7.0, device="cuda")
    lib.train_step(field, geom, 0, torch.empty(0, dtype=torch.int32, device="cuda"),
                   torch.empty(0, device="cuda"), 16, loss_t, ws)
    assert _np(loss_t)[0] == 0.0
    assert np.array_equal(_np(field.flat_params()), flat)
    miss = np.setdiff1d(np.arange(GEOM.det_nu * GEOM.det_nv), hit_pixels(GEOM, 0))[:50].astype(np.int32)
    ws = lib.workspace(lib.step_workspace_bytes(field, len(miss), 16))
    a = torch.full((len(miss),), 5.0, device="cuda")
    lib.render_forward(field, geom, 0, _t(miss), 16, a, ws)
    assert np.all(_np(a) == 0.0)


def test_nonfinite_measurement_skips_the_step(lib):
    cfg = field_cfg()
    flat = S.init_params(cfg, 9).astype(np.float32)
    field = lib.Field(cfg, params=flat)
    geom = lib.Geometry.from_config(GEOM)
    pix = batch(GEOM, 0, 64, seed=1)
    a_meas = np.zeros(64, dtype=np.float32)
    a_meas[5] = np.nan
    ws = lib.workspace(lib.step_workspace_bytes(field, 64, 16))
    loss_t = torch.zeros(1, device="cuda")
    lib.train_step(field, geom, 0, _t(pix), _t(a_meas), 16, loss_t, ws)
    flags, _, step = field.poll_status()
    assert flags & lib.FLAG_NONFINITE and flags & lib.FLAG_SKIPPED and step == 0
    assert np.array_equal(_np(field.flat_params()), flat)
    a_meas[5] = 0.1
    lib.train_step(field, geom, 0, _t(pix), _t(a_meas), 16, loss_t, ws)
    flags, _, step = field.poll_status()
    assert flags == 0 and step == 1


def test_f16_dynamic_loss_scale_halves_on_overflow_and_grows_back(lib):
    """Dynamic loss scaling of the FP16 path: a scale of 2^40 overflows the 16-bit
    backward (non-finite dL/dh), so the step is skipped, the parameters stay as they
    were and the scale halves, until a scale fits; a safe scale doubles after every
    growth_interval applied steps."""
    geom = lib.Geometry.from_config(GEOM)
    pix = batch(GEOM, 0, 128, seed=2)
    a_meas = np.random.default_rng(2).uniform(0, 0.8, size=len(pix)).astype(np.float32)
    N = 48
    cfg = field_cfg(precision=S.PREC_F16, loss_scale_init=2.0 ** 40, growth_interval=3)
    flat = S.init_params(cfg, 12).astype(np.float32)
    field = lib.Field(cfg, params=flat)
    ws = lib.workspace(lib.step_workspace_bytes(field, len(pix), N))
    loss_t = torch.zeros(1, device="cuda")
    scale, skipped = 2.0 ** 40, 0
    for _ in range(60):
        lib.train_step(field, geom, 0, _t(pix), _t(a_meas), N, loss_t, ws)
        flags, s, step = field.poll_status()
        if not flags & lib.FLAG_SKIPPED:
            assert flags == 0 and step == 1 and s == scale
            break
        assert flags & lib.FLAG_NONFINITE and step == 0 and s == scale / 2
        assert np.array_equal(_np(field.flat_params()), flat)
        assert float(field.grads.abs().max()) == 0.0
        scale, skipped = s, skipped + 1
    else:
        raise AssertionError("the loss scale never came down to a finite step")
    assert skipped >= 3 and scale == 2.0 ** (40 - skipped)
    assert np.isfinite(_np(loss_t)[0])

    cfg = replace(cfg, loss_scale_init=1024.0)
    field = lib.Field(cfg, params=flat)
    for k in range(1, 7):
        lib.train_step(field, geom, 0, _t(pix), _t(a_meas), N, loss_t, ws)
        flags, s, step = field.poll_status()
        assert flags == 0 and step == k
        assert s == 1024.0 * 2 ** (k // 3)


def test_argument_errors_are_reported(lib):
    cfg = field_cfg()
    field = lib.Field(cfg, params=S.init_params(cfg, 0))
    geom = lib.Geometry.from_config(GEOM)
    pix = _t(batch(GEOM, 0, 8, seed=0))
    small = lib.workspace(16)
    with pytest.raises(lib.NHError) as e:
        lib.render_forward(field, geom, 0, pix, 16, torch.empty(8, device="cuda"), small)
    assert e.value.status == -3
    with pytest.raises(lib.NHError) as e:
        lib.render_forward(field, geom, 99, pix, 16, torch.empty(8, device="cuda"), lib.workspace(1 << 16))
    assert e.value.status == -1
    with pytest.raises(lib.NHError) as e:
        lib.Field(replace(cfg, width=64))
    assert e.value.status == -6


# ------------------------------------------------------------------------------ full sizes
@pytest.mark.parametrize("wname", ["paper_fp32", "large_bf16"])
def test_full_size_sampled_rays_match_oracle(lib, wname):
    """The configuration the benchmark times, checked on sampled rays: the forward of
    every ray runs, the oracle recomputes 6 of them; the backward of two single rays
    (one-hot dL/dA) is compared on the dense parameters and the touched table rows."""
    w = S.WORKLOADS[wname]
    cfg = replace(w.field, precision=S.PREC_F32) if w.field.precision == S.PREC_F32 else w.field
    flat = S.init_params(cfg, 1, table_scale=0.5).astype(np.float32)
    field = lib.Field(cfg, params=flat)
    geom = lib.Geometry.from_config(w.geometry)
    og = oracle_geom(w.geometry)
    rng = np.random.default_rng(0)
    view = 3
    pix = rng.choice(hit_pixels(w.geometry, view), size=w.n_rays, replace=False).astype(np.int32)
    N = w.n_samples
    ws = lib.workspace(lib.step_workspace_bytes(field, len(pix), N))
    a = torch.empty(len(pix), device="cuda")
    lib.render_forward(field, geom, view, _t(pix), N, a, ws)
    ref_flat = rounded_tables(flat, cfg, cfg.precision).astype(np.float64)
    pick = rng.choice(len(pix), size=6, replace=False)
    ref = oracle.render(ref_flat, cfg, og, view, pix[pick], N)
    tol_f, tol_g = MIXED_TOL.get(cfg.precision, (1e-5, 1e-3))
    if cfg.precision == S.PREC_F32:
        np.testing.assert_allclose(_np(a)[pick], ref, rtol=1e-5, atol=1e-6)
    else:
        assert np.abs(_np(a)[pick] - ref).max() <= tol_f * np.abs(ref).max()
    for r in pick[:2]:
        field.grads.zero_()
        dLdA = np.zeros(len(pix), dtype=np.float32)
        dLdA[r] = 1.0
        lib.render_backward(field, geom, view, _t(pix), N, _t(dLdA), ws)
        A, cache = oracle.render_forward(ref_flat, cfg, og, view, pix[r:r + 1], N)
        g_ref = oracle.render_backward(cache, np.array([1.0]), cfg)
        if cfg.precision == S.PREC_F32:
            _grad_close(_np(field.flat_grads()), g_ref, cfg, what=f"{wname} ray {r}")
        else:
            _grad_close(_np(field.flat_grads()), g_ref, cfg, what=f"{wname} ray {r}", norm_rtol=tol_g)


@pytest.mark.parametrize("wname", ["paper_fp32", "paper_bf16"])
def test_full_size_fused_step_matches_oracle(lib, wname):
    """The launch the benchmark times (accumulate_step: the fused kernel on 2048 rays
    x 192 samples of the paper workload's field) against the oracle on the whole
    batch: the loss within 1e-5 (FP32) or the mixed forward bound, every gradient
    group within 1e-3 of its largest entry (FP32, with the ReLU-kink allowance on
    the table entries that ambiguous samples reach) or the mixed norm bound."""
    w = S.WORKLOADS[wname]
    cfg = w.field
    flat = S.init_params(cfg, 1, table_scale=0.5).astype(np.float32)
    field = lib.Field(cfg, params=flat)
    geom = lib.Geometry.from_config(w.geometry)
    og = oracle_geom(w.geometry)
    rng = np.random.default_rng(0)
    view = 3
    pix = rng.choice(hit_pixels(w.geometry, view), size=w.n_rays, replace=False).astype(np.int32)
    a_meas = rng.uniform(0.0, 0.8, size=len(pix)).astype(np.float32)
    N = w.n_samples
    ws = lib.workspace(lib.step_workspace_bytes(field, len(pix), N))
    loss_t = torch.zeros(1, device="cuda")
    lib.accumulate_step(field, geom, view, _t(pix), _t(a_meas), N, loss_t, ws)
    info = lib.launch_info()
    assert info["grid"] > 0 and info["tmem_cols"] == 256          # the fused kernel ran
    ref_flat = rounded_tables(flat, cfg, cfg.precision).astype(np.float64)
    A, cache = oracle.render_forward(ref_flat, cfg, og, view, pix, N)
    ref_loss, dLdA = oracle.loss_and_grad(A, a_meas, S.LOSS_MSE)
    g_ref = oracle.render_backward(cache, dLdA, cfg)
    g = _np(field.flat_grads()) / cfg.loss_scale_init
    if cfg.precision == S.PREC_F32:
        assert abs(_np(loss_t)[0] - ref_loss) <= 1e-5 * ref_loss
        bad = fp32_gradient_errors(g, g_ref, cfg, cache, dLdA)
        assert not bad, (f"{wname} full batch", bad)
    else:
        tol_f, tol_g = MIXED_TOL[cfg.precision]
        assert abs(_np(loss_t)[0] - ref_loss) <= 2 * tol_f * ref_loss
        _grad_close(g, g_ref, cfg, what=f"{wname} full batch", norm_rtol=tol_g)


# ------------------------------------------------------------------------------ FFT channel mask
def test_fft_channel_mask_matches_oracle(lib):
    """The channel mask chosen from the library's gather on the GPU (Sec. 2.3) equals
    the oracle's, on a planted field (a smooth dense level, constant levels, a
    white-noise hashed level) and on a randomly initialised 16-level field."""
    from paper_2506_19742_gb300 import channel_mask as cm
    cfg = S.FieldConfig(n_levels=8, n_feat=2, log2_T=10, base_res=4, max_res=512, norm=S.NORM_LN,
                        hidden_layers=1, width=32)
    assert oracle.level_resolutions(8, 4, 512)[0] == 4
    flat = S.init_params(cfg, 0).astype(np.float32)
    T = cfg.T
    tab = np.zeros((8, T, 2), dtype=np.float32)   # levels 1..6 constant (no variance: kept)
    for zz in range(5):
        for yy in range(5):
            for xx in range(5):
                tab[0, xx + 5 * yy + 25 * zz] = [0.3 * xx - 0.1 * zz, 0.2 * yy]
    tab[7] = np.random.default_rng(1).normal(size=(T, 2))
    flat[: 8 * T * 2] = tab.ravel()
    cases = [(cfg, flat, 32), (field_cfg(n_levels=16, log2_T=12, base_res=16, max_res=512),
                               S.init_params(field_cfg(n_levels=16, log2_T=12, base_res=16, max_res=512), 3,
                                             table_scale=0.5), 24)]
    masks = []
    for c, f, G in cases:
        field = lib.Field(c, params=f)
        mask, frac = cm.select_channel_mask(field, G=G, cutoff=0.25, threshold=0.85)
        ref_mask, ref_frac = oracle.channel_mask(f.astype(np.float64), c, G=G, cutoff=0.25, threshold=0.85)
        np.testing.assert_allclose(frac, ref_frac, rtol=0, atol=1e-5)
        clear = np.abs(ref_frac - 0.85) > 1e-4            # decisions float32 rounding cannot flip
        assert np.array_equal(mask[clear], ref_mask[clear].astype(np.float32)), (frac, ref_frac)
        masks.append(mask)
    np.testing.assert_array_equal(masks[0], [1] * 14 + [0, 0])


@pytest.mark.parametrize("precision,G", [(S.PREC_BF16, 33), (S.PREC_F32, 64)])
def test_fft_channel_mask_selection_through_the_c_abi(lib, precision, G):
    """field_select_channel_mask (Sec. 2.3) on the paper-scale field shape (L16 F2
    16..2048, one LN; 2^16 entries per level): every channel's high-frequency
    fraction within 1e-5 of the oracle's (tables rounded as the library stores
    them), the mask equal wherever float32 feature rounding cannot flip the
    decision, an odd grid (33^3) and the read-out grid (64^3), the same bits on a
    second call, and the mask installed in the field only when asked."""
    cfg = replace(S.WORKLOADS["paper_fp32"].field, precision=precision, log2_T=16)
    flat = S.init_params(cfg, 17, table_scale=1.0).astype(np.float32)
    tab = flat[: cfg.n_levels * cfg.T * 2].reshape(cfg.n_levels, cfg.T, 2)
    tab[3] = 0.0                                      # a zero level: no variance, fraction 0
    field = lib.Field(cfg, params=flat)
    D = cfg.d_in
    ws = lib.workspace(lib.channel_mask_workspace_bytes(field, G))
    frac = torch.empty(D, dtype=torch.float64, device="cuda")
    mask = torch.empty(D, device="cuda")
    lib.select_channel_mask(field, G, 0.25, 0.85, False, frac, mask, ws)
    torch.cuda.synchronize()
    f1, m1 = _np(frac).copy(), _np(mask).copy()
    assert np.all(_np(field.state)[16:16 + D] == 1.0)            # not installed
    lib.select_channel_mask(field, G, 0.25, 0.85, True, frac, mask, ws)
    torch.cuda.synchronize()
    assert np.array_equal(_np(frac), f1) and np.array_equal(_np(mask), m1)
    assert np.array_equal(_np(field.state)[16:16 + D], m1)        # installed
    ref_mask, ref_frac = oracle.channel_mask(rounded_tables(flat, cfg, precision).astype(np.float64), cfg, G=G,
                                             cutoff=0.25, threshold=0.85)
    print(np.round(f1, 4))
    np.testing.assert_allclose(f1, ref_frac, rtol=0, atol=1e-5)
    assert f1[6] == 0.0 and f1[7] == 0.0
    clear = np.abs(ref_frac - 0.85) > 1e-4
    assert np.array_equal(m1[clear], ref_mask[clear].astype(np.float32))
    assert 0 < m1.sum() < D                                      # both decisions occur


# ------------------------------------------------------------------------------ stored record
def test_library_matches_the_stored_oracle_step(lib):
    """The library against tests/golden/oracle_step.json (the oracle's record of one
    seeded step): A and the loss within 1e-5, the recorded gradient entries within
    1e-3 of the largest gradient, and, where the gradient is not tiny, the entries
    after one Adam step."""
    import json
    import os
    import sys
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    sys.path.insert(0, here)
    import make_golden
    ref = json.load(open(os.path.join(here, "oracle_step.json")))
    _, flat, pix, a_meas = make_golden.case()
    cfg, N, view = make_golden.FIELD, make_golden.N, make_golden.VIEW
    assert pix.tolist() == ref["pix"]
    field = lib.Field(cfg, params=flat.astype(np.float32))
    geom = lib.Geometry.from_config(make_golden.GEOM)
    ws = lib.workspace(lib.step_workspace_bytes(field, len(pix), N))
    a = torch.empty(len(pix), device="cuda")
    lib.render_forward(field, geom, view, _t(pix), N, a, ws)
    np.testing.assert_allclose(_np(a), ref["A"], rtol=1e-5, atol=1e-7)
    loss_t = torch.zeros(1, device="cuda")
    lib.accumulate_step(field, geom, view, _t(pix), _t(a_meas), N, loss_t, ws)
    assert abs(_np(loss_t)[0] - ref["loss"]) <= 1e-5 * ref["loss"]
    g = _np(field.flat_grads())[ref["grad_index"]]
    assert np.abs(g - np.array(ref["grad_value"])).max() <= 1e-3 * ref["grad_max"]
    lib.optimizer_step(field)
    p = _np(field.flat_params())[ref["grad_index"]]
    big = np.abs(np.array(ref["grad_value"])) > 1e-2 * ref["grad_max"]   # step sign not decided by rounding
    assert big.sum() >= 8
    np.testing.assert_allclose(p[big], np.array(ref["param_after_adam"])[big], rtol=0, atol=2e-6)


def test_many_short_rays_fill_every_loss_partial(lib):
    """A batch larger than the grid holds at once: 20000 rays of 8 samples (one chunk,
    8 rays per CTA, 2500 ray groups over the persistent CTAs) gives the oracle's loss
    and gradient."""
    cfg = field_cfg(n_levels=8, hidden_layers=2, log2_T=12)
    flat = S.init_params(cfg, 43, table_scale=0.5).astype(np.float32)
    field = lib.Field(cfg, params=flat)
    g = S.GeometryConfig(n_views=6, det_nu=200, det_nv=200)
    geom = lib.Geometry.from_config(g)
    og = oracle_geom(g)
    pix = batch(g, 1, 20000, seed=5)
    N = 8
    a_meas = np.random.default_rng(3).uniform(0, 0.8, size=len(pix)).astype(np.float32)
    A, cache = oracle.render_forward(flat.astype(np.float64), cfg, og, 1, pix, N)
    ref_loss, dLdA = oracle.loss_and_grad(A, a_meas, S.LOSS_MSE)
    ws = lib.workspace(lib.step_workspace_bytes(field, len(pix), N))
    loss_t = torch.zeros(1, device="cuda")
    lib.accumulate_step(field, geom, 1, _t(pix), _t(a_meas), N, loss_t, ws)
    assert abs(_np(loss_t)[0] - ref_loss) <= 1e-5 * ref_loss
    _grad_close(_np(field.flat_grads()), oracle.render_backward(cache, dLdA, cfg), cfg, what="many rays")
