"""Property-based pins of the oracle (CPU, hypothesis): invariants that hold for
any input, so that a slip in a rarely hit branch (a clamp, a boundary cell, a
dense/hashed switch, a loss kink) still fails somewhere."""
import math

import numpy as np
import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import example, given, settings  # noqa: E402
from hypothesis import strategies as st  # noqa: E402

import oracle  # noqa: E402
import synthetic as S  # noqa: E402

coord = st.floats(min_value=-0.25, max_value=1.25, allow_nan=False, width=32)
points = st.lists(st.tuples(coord, coord, coord), min_size=1, max_size=40)


@settings(max_examples=60, deadline=None, derandomize=True, database=None)
@given(points, st.integers(min_value=1, max_value=600), st.integers(min_value=4, max_value=16))
@example([(0.0, 0.0, float(np.float32(0.9)))], 50, 4)
def test_corners_stay_in_range_and_weights_partition_unity(pts, n, log2T):
    """For any point (clamped to the cube) and resolution: weights in [0, 1] summing
    to 1, every index below T (below (N+1)^3 on a dense level), and the cell's
    corner 0 at the floor of the float32 position x N (capped at N - 1)."""
    x = np.array(pts, dtype=np.float32)
    T = 1 << log2T
    idx, w, fr = oracle.corners(x, [n], T)
    assert np.all(w >= 0.0) and np.all(w <= 1.0)
    np.testing.assert_allclose(w.sum(axis=-1), 1.0, rtol=0, atol=1e-12)
    bound = (n + 1) ** 3 if (n + 1) ** 3 <= T else T
    assert np.all(idx < bound)
    assert np.all(fr >= 0.0) and np.all(fr <= 1.0)
    # the position x N is taken in float32 (as on the GPU): its float32 value, not
    # the exact product, picks the cell (0.9f * 50 rounds up to 45 exactly)
    p = np.clip(x, 0.0, 1.0) * np.float32(n)
    c = np.minimum(np.floor(p.astype(np.float64)), n - 1)
    np.testing.assert_allclose(c + fr[:, 0, :], p, rtol=0, atol=1e-5 * n)


@settings(max_examples=40, deadline=None, derandomize=True, database=None)
@given(st.lists(st.floats(min_value=-5, max_value=5, allow_nan=False), min_size=16, max_size=16),
       st.floats(min_value=1e-6, max_value=3.0))
def test_layer_norm_output_moments_for_any_row(vals, scale):
    """One LayerNorm group: the normalized row has mean 0 and variance s2 / (s2 + eps)."""
    cfg = S.FieldConfig(n_levels=8, n_feat=2, norm=S.NORM_LN)
    h = np.array(vals, dtype=np.float64)[None, :] * scale
    D = 16
    y, _ = oracle.normalize_forward(h, np.ones(D), np.zeros(D), np.ones(D), cfg)
    s2 = h.var()
    assert abs(y.mean()) < 1e-9
    assert abs(y.var() - s2 / (s2 + cfg.ln_eps)) < 1e-9


@settings(max_examples=60, deadline=None, derandomize=True, database=None)
@given(st.lists(st.tuples(st.floats(0, 2, allow_nan=False), st.floats(0, 2, allow_nan=False)),
                min_size=1, max_size=30))
def test_losses_are_means_and_gradients_are_their_derivatives(pairs):
    """MSE and L1 over any batch: the value is the mean, and the gradient is the
    derivative of the mean (sign(0) = 0 for L1)."""
    A = np.array([p[0] for p in pairs])
    Am = np.array([p[1] for p in pairs])
    R = len(A)
    l, g = oracle.loss_and_grad(A, Am, S.LOSS_MSE)
    assert math.isclose(l, float(np.mean((A - Am) ** 2)), rel_tol=1e-12, abs_tol=1e-15)
    np.testing.assert_allclose(g, 2 * (A - Am) / R, rtol=1e-12, atol=1e-15)
    l, g = oracle.loss_and_grad(A, Am, S.LOSS_L1)
    assert math.isclose(l, float(np.mean(np.abs(A - Am))), rel_tol=1e-12, abs_tol=1e-15)
    np.testing.assert_allclose(g, np.sign(A - Am) / R, rtol=0, atol=0)


@settings(max_examples=40, deadline=None, derandomize=True, database=None)
@given(st.integers(min_value=0, max_value=2 ** 40), st.integers(min_value=1, max_value=64),
       st.lists(st.integers(min_value=0, max_value=1 << 20), min_size=1, max_size=8))
def test_stratum_offsets_lie_in_their_stratum_for_any_seed(seed, N, pix):
    """Any seed and pixels: offsets in [0, 1), exact multiples of 2^-24, the same for
    the same (seed, pixel, sample), and 1/2 for seed 0."""
    pix = np.array(pix, dtype=np.int32)
    u = oracle.stratum_offsets(seed, pix, N)
    assert u.shape == (len(pix), N) and u.dtype == np.float32
    assert np.all(u >= 0.0) and np.all(u < 1.0)
    if seed == 0:
        assert np.all(u == np.float32(0.5))
    else:
        k = u.astype(np.float64) * 2.0 ** 24
        assert np.all(k == np.floor(k))
        np.testing.assert_array_equal(u[0], oracle.stratum_offsets(seed, pix[:1], N)[0])


@settings(max_examples=25, deadline=None, derandomize=True, database=None)
@given(st.integers(min_value=11, max_value=14), st.integers(min_value=0, max_value=2 ** 32 - 1),
       st.floats(min_value=0.0, max_value=1.0), st.floats(min_value=0.0, max_value=1.0))
def test_ssim_is_symmetric_bounded_and_one_only_for_equal_volumes(D, seed, a, noise):
    """Any pair of volumes in [0, 1]: the local index is symmetric in its two
    volumes and lies in [-1, 1]. A volume against itself scores 1 at every window.
    An affine copy a x + (1 - a) / 2 (a > 0) keeps the structure term at 1, so the
    index equals the product of the luminance and contrast terms, each <= 1."""
    rng = np.random.default_rng(seed)
    x = rng.random((D, D, D))
    y = np.clip(x + noise * rng.standard_normal((D, D, D)), 0.0, 1.0)
    m = oracle.ssim_map(x, y)
    np.testing.assert_allclose(m, oracle.ssim_map(y, x), rtol=0, atol=1e-14)
    assert np.all(m <= 1.0 + 1e-12) and np.all(m >= -1.0 - 1e-12)
    np.testing.assert_allclose(oracle.ssim_map(x, x), 1.0, rtol=0, atol=1e-12)
    if a > 1e-3:
        z = a * x + (1.0 - a) / 2.0
        mz = oracle.ssim_map(x, z)
        assert np.all(mz <= 1.0 + 1e-12)
        if abs(a - 1.0) > 1e-3:
            assert np.all(mz < 1.0)
