"""Rendering, losses, Adam and the training / pre-training steps (oracle).

Test infrastructure: only the tests, the smoke check and the benchmark's CPU legs
use it.

* Beer-Lambert ray sum (Sec. 2.2, Eq. 1): A = -ln(I / I0) = sum_i mu_i delta_i,
  accumulated in float64; a ray that misses the volume has A = 0.
* Pixel loss (Sec. 2.5, Eq. 3) is an L1 norm of A_gt - sum_i M(x_i) delta_i; the
  benchmark's workloads use the squared error instead. Both are provided and
  read as a mean over the R rays of the batch:
  MSE = (1/R) sum (A - A_meas)^2,   L1 = (1/R) sum |A - A_meas|, sign(0) = 0.
* Voxel loss of Mapping Consistency Initialization (Sec. 2.4, Eq. 2):
  (1/P) sum |mu_gt - M(x)| over P sampled voxel centres, sign(0) = 0.
* Adam (Sec. 3.1, learning rate 1e-3; Kingma & Ba): torch's defaults
  beta = (0.9, 0.999), eps = 1e-8, bias correction, no weight decay, applied
  densely to every parameter each step (entries no ray touched still decay
  their moments). With a loss scale S, gradients are divided by S first; a
  non-finite gradient skips the step.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from .geometry import ray_setup, sample_points, stratum_offsets, voxel_centres_f32
from .field import unflatten, flatten, field_forward, field_backward


@dataclasses.dataclass
class AdamState:
    m: np.ndarray
    v: np.ndarray
    t: int = 0

    @classmethod
    def zeros(cls, n):
        return cls(np.zeros(n), np.zeros(n), 0)


def render_forward(flat, cfg, geom, view, pix, N, mask=None, jitter_seed=0):
    """Predicted projections A (R,) of rays (view, pix). geom = (tab, du, dv, nu, nv).
    jitter_seed 0: midpoint samples; otherwise stratified jitter (stratum_offsets)."""
    tab, du, dv, nu, nv = geom
    p = unflatten(flat, cfg)
    o, d, near, far, hit = ray_setup(tab, du, dv, nu, nv, view, pix)
    u = stratum_offsets(jitter_seed, pix, N) if jitter_seed else None
    x, delta = sample_points(o, d, near, far, N, u)
    R = len(pix)
    A = np.zeros(R)
    xh = x[hit].reshape(-1, 3)
    if xh.shape[0] == 0:
        return A, (p, None, hit, delta, N)
    mu, cache = field_forward(p, xh, cfg, mask)
    A[hit] = (mu.reshape(-1, N) * delta[hit].astype(np.float64)[:, None]).sum(axis=1)
    return A, (p, cache, hit, delta, N)


def render(flat, cfg, geom, view, pix, N, mask=None, jitter_seed=0):
    """Eq. 1 for each ray of the batch."""
    return render_forward(flat, cfg, geom, view, pix, N, mask, jitter_seed)[0]


def loss_and_grad(A, A_meas, kind):
    """Batch loss and dL/dA. kind 0 = mean squared error, 1 = mean absolute error (Eq. 3)."""
    r = A - np.asarray(A_meas, dtype=np.float64)
    R = len(r)
    if kind == 0:
        return float(np.mean(r * r)), 2.0 * r / R
    return float(np.mean(np.abs(r))), np.sign(r) / R


def render_backward(cache, dLdA, cfg):
    """Flat gradient of sum_r dLdA_r * A_r with respect to every parameter."""
    p, fcache, hit, delta, N = cache
    if fcache is None:
        g = {k: (np.zeros_like(v) if not isinstance(v, list) else [np.zeros_like(a) for a in v])
             for k, v in p.items()}
        return flatten(g)
    dmu = (np.asarray(dLdA, dtype=np.float64)[hit] * delta[hit].astype(np.float64))
    dmu = np.repeat(dmu, N)
    return flatten(field_backward(p, fcache, dmu, cfg))


def adam_step(flat, grad, state, cfg, loss_scale=1.0):
    """One Adam update. Returns (new params, new state, skipped)."""
    g = np.asarray(grad, dtype=np.float64) / loss_scale
    if not np.all(np.isfinite(g)):
        return np.asarray(flat, dtype=np.float64), state, True
    t = state.t + 1
    m = cfg.beta1 * state.m + (1.0 - cfg.beta1) * g
    v = cfg.beta2 * state.v + (1.0 - cfg.beta2) * g * g
    mhat = m / (1.0 - cfg.beta1 ** t)
    vhat = v / (1.0 - cfg.beta2 ** t)
    new = np.asarray(flat, dtype=np.float64) - cfg.lr * mhat / (np.sqrt(vhat) + cfg.adam_eps)
    return new, AdamState(m, v, t), False


def train_step(flat, state, cfg, geom, view, pix, A_meas, N, mask=None, jitter_seed=0):
    """One reconstruction step (Sec. 2.5): render, loss, backward, Adam."""
    A, cache = render_forward(flat, cfg, geom, view, pix, N, mask, jitter_seed)
    loss, dLdA = loss_and_grad(A, A_meas, cfg.loss)
    grad = render_backward(cache, dLdA, cfg)
    new, state, _ = adam_step(flat, grad, state, cfg)
    return new, state, loss, grad


def fit_points_step(flat, state, cfg, xyz, mu_gt, mask=None, adam=True):
    """One voxel-loss pre-training step (Sec. 2.4, Eq. 2) on points xyz (P, 3) f32."""
    p = unflatten(flat, cfg)
    mu, cache = field_forward(p, np.asarray(xyz, dtype=np.float32), cfg, mask)
    r = mu - np.asarray(mu_gt, dtype=np.float64)
    P = len(r)
    loss = float(np.mean(np.abs(r)))
    grad = flatten(field_backward(p, cache, np.sign(r) / P, cfg))
    if not adam:
        return flat, state, loss, grad
    new, state, _ = adam_step(flat, grad, state, cfg)
    return new, state, loss, grad


def query_points(flat, cfg, xyz, mask=None):
    """mu = M(x) at the given points."""
    mu, _ = field_forward(unflatten(flat, cfg), np.asarray(xyz, dtype=np.float32), cfg, mask)
    return mu


def query_volume(flat, cfg, D, mask=None):
    """mu at the D^3 voxel centres, shape (D, D, D) [z][y][x] (the M(x, y, z) of Eq. 2)."""
    return query_points(flat, cfg, voxel_centres_f32(D), mask).reshape(D, D, D)
