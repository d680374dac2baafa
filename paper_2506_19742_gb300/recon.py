"""Reconstruction loop and Mapping Consistency Initialization on the C ABI.

``Reconstruction`` trains one field from cone-beam projections with train_step
(Sec. 2.5) and evaluates it with query_volume / volume_mse (PSNR, Sec. 3.2);
``train_to_psnr`` runs it until PSNR targets are reached and reports steps and
GPU seconds of training (evaluation excluded). ``pretrain_mci`` is the voxel-loss
pre-training of Sec. 2.1 / 2.4 (Eq. 2): one shared LN + MLP is fitted to several
attenuation volumes, each case keeping its own hash tables; ``transfer`` loads only
the LN and MLP weights into a new field (Sec. 2.1). Every step runs in the
library's kernels; this module only orders calls and moves batches.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import nhcbct as nh

LN_MLP = nh.PART_LN | nh.PART_MLP


class Reconstruction:
    """One field being reconstructed from projections of one scan geometry."""

    def __init__(self, cfg, geom: "nh.Geometry", params=None, device="cuda"):
        self.cfg, self.geom, self.device = cfg, geom, device
        self.field = nh.Field(cfg, device=device, params=params)
        self.loss = torch.zeros(1, device=device)
        self._ws = None
        self._ws_key = None
        self.steps = 0

    def _workspace(self, R, N):
        if self._ws_key != (R, N):
            self._ws = nh.workspace(nh.step_workspace_bytes(self.field, R, N), self.device)
            self._ws_key = (R, N)
        return self._ws

    def step(self, view, pix, a_meas, n_samples, jitter_seed=0):
        """One training step on device-resident pix (int32) / a_meas (float32);
        jitter_seed 0 samples at stratum midpoints, any other value jitters them."""
        nh.train_step(self.field, self.geom, view, pix, a_meas, n_samples, self.loss,
                      self._workspace(pix.numel(), n_samples), jitter_seed=jitter_seed)
        self.steps += 1

    def volume(self, D):
        out = torch.empty(D ** 3, device=self.device)
        nh.query_volume(self.field, D, out)
        return out

    def psnr(self, vol_gt):
        """PSNR (data range 1) of the field at the D^3 voxel centres of vol_gt (D^3 floats)."""
        D = int(round(vol_gt.numel() ** (1.0 / 3.0)))
        return nh.psnr(self.volume(D), vol_gt.reshape(-1))

    def ssim(self, vol_gt):
        """3-D SSIM (data range 1) of the field at the D^3 voxel centres of vol_gt."""
        D = int(round(vol_gt.numel() ** (1.0 / 3.0)))
        return nh.ssim(self.volume(D), vol_gt.reshape(-1))


def train_to_psnr(rec: Reconstruction, batches, n_samples, vol_gt, targets=(30.0, 35.0), eval_every=50,
                  max_steps=3000):
    """Trains until every target PSNR is reached or max_steps. ``batches`` yields
    (view, pix, a_meas) device tensors forever. Returns steps and training seconds
    (CUDA events around the steps only) at which each target was first reached
    (None if not), and the PSNR curve."""
    stream = torch.cuda.current_stream()
    reached = {t: None for t in targets}
    curve = []
    train_ms = 0.0
    it = iter(batches)
    step = 0
    while step < max_steps:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(min(eval_every, max_steps - step)):
            view, pix, a = next(it)
            rec.step(view, pix, a, n_samples)
            step += 1
        e1.record(stream)
        e1.synchronize()
        train_ms += e0.elapsed_time(e1)
        p = rec.psnr(vol_gt)
        curve.append((step, round(train_ms / 1e3, 4), round(p, 3)))
        for t in targets:
            if reached[t] is None and p >= t:
                reached[t] = (step, train_ms / 1e3)
        if all(v is not None for v in reached.values()):
            break
    best = max(c[2] for c in curve) if curve else float("nan")
    return {"steps_to": {str(t): (v[0] if v else None) for t, v in reached.items()},
            "seconds_to": {str(t): (round(v[1], 4) if v else None) for t, v in reached.items()},
            "final_psnr": curve[-1][2] if curve else float("nan"), "best_psnr": best,
            "steps": step, "train_seconds": round(train_ms / 1e3, 4), "curve": curve}


def pretrain_mci(cfg, volumes, steps, points_per_step, seed=0, device="cuda"):
    """Voxel-loss pre-training (Eq. 2) of one LN + MLP shared by several cases.

    ``volumes``: list of D^3 float32 CUDA tensors (attenuation fields, [z][y][x]).
    Case c keeps its own hash tables in its own field; before each of its steps the
    shared LN + MLP weights and their Adam moments are imported, and afterwards
    exported back. Points are P random voxel centres of the case. Returns the
    shared LN + MLP parameters (export of NH_PART_LN | NH_PART_MLP) and the loss
    curve."""
    rng = np.random.default_rng(seed)
    fields = [nh.Field(cfg, device=device, params=_init(cfg, seed + 1000 + c)) for c in range(len(volumes))]
    shared = fields[0].export(LN_MLP | nh.PART_ADAM)
    ws = nh.workspace(nh.points_workspace_bytes(fields[0], points_per_step), device)
    loss = torch.zeros(1, device=device)
    curve = []
    for s in range(steps):
        c = s % len(volumes)
        f = fields[c]
        vol = volumes[c]
        D = int(round(vol.numel() ** (1.0 / 3.0)))
        idx = rng.integers(0, D ** 3, size=points_per_step)
        z, rem = np.divmod(idx, D * D)
        y, x = np.divmod(rem, D)
        xyz = ((np.stack([x, y, z], axis=-1) + 0.5) / D).astype(np.float32)
        xyz_d = torch.from_numpy(xyz).to(device)
        mu = vol.reshape(-1)[torch.from_numpy(idx).to(device)].contiguous()
        f.import_(LN_MLP | nh.PART_ADAM, shared)
        nh.fit_points_step(f, xyz_d, mu, loss, ws)
        shared = f.export(LN_MLP | nh.PART_ADAM)
        if s % max(1, steps // 20) == 0 or s == steps - 1:
            curve.append((s, float(loss.item())))
    n = fields[0].export_bytes(LN_MLP) // 4
    return shared[:n].clone(), curve


def transfer(params_ln_mlp, field):
    """Mapping Consistency Initialization: load only the LN and MLP weights (Sec. 2.1)."""
    field.import_(LN_MLP, params_ln_mlp)


def _init(cfg, seed):
    """Float32 initial parameters: tables U(-1e-4, 1e-4), gamma 1, beta 0, Linear default."""
    rng = np.random.default_rng(seed)
    L, F, T, D, W, H = cfg.n_levels, cfg.n_feat, 1 << cfg.log2_T, cfg.n_levels * cfg.n_feat, cfg.width, \
        cfg.hidden_layers
    parts = [rng.uniform(-1e-4, 1e-4, size=L * T * F), np.ones(D), np.zeros(D)]
    dims = [D] + [W] * H + [1]
    for k in range(H + 1):
        b = 1.0 / math.sqrt(dims[k])
        parts += [rng.uniform(-b, b, size=dims[k + 1] * dims[k]), rng.uniform(-b, b, size=dims[k + 1])]
    return np.concatenate(parts).astype(np.float32)
