"""FFT channel masking of the hash features (Sec. 2.3).

Some channels of the hash features carry noise rather than structure; the paper
tells them apart with a Fast Fourier Transform and masks them during training, but
gives no grid, statistic or threshold. This module takes the following reading:

- every channel of the hash features h (the gather's output, before
  normalization) is evaluated by the library's gather (``encode_points``) at the
  voxel centres (k + 1/2) / G of a G^3 grid over the volume, the grid on which the
  reconstruction is read out;
- each channel's mean is removed and its 3-D power spectrum taken (cuFFT through
  torch.fft);
- the channel's high-frequency fraction is the share of that power at radial
  frequencies |k| > cutoff, in cycles per voxel (|k| <= sqrt(3) / 2);
- a channel whose fraction exceeds the threshold is noise-like and gets mask 0
  (``field_set_channel_mask``); all others keep 1.

White noise puts about 0.93 of its power beyond a cutoff of 1/4, a smooth field
almost none. The selection is an occasional step between training steps, not
part of the step itself; the mask multiply inside the training kernels is.
"""
from __future__ import annotations

import numpy as np
import torch

from . import nhcbct as nh


def voxel_grid(G: int) -> np.ndarray:
    """(G^3, 3) float32 voxel centres (k + 1/2) / G, flattened [z][y][x]."""
    c = (np.arange(G, dtype=np.float32) + np.float32(0.5)) / np.float32(G)
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=-1).astype(np.float32)


def high_frequency_fraction(h: torch.Tensor, G: int, cutoff: float) -> torch.Tensor:
    """Per channel of h (G^3, C), [z][y][x] order: share of the mean-free power
    spectrum at |k| > cutoff (0 for a channel without variance)."""
    h = h.reshape(G, G, G, -1).to(torch.float64)
    h = h - h.mean(dim=(0, 1, 2), keepdim=True)
    P = torch.fft.fftn(h, dim=(0, 1, 2)).abs().square()
    f = torch.fft.fftfreq(G, device=h.device, dtype=torch.float64)
    kz, ky, kx = torch.meshgrid(f, f, f, indexing="ij")
    high = (kx * kx + ky * ky + kz * kz).sqrt() > cutoff
    tot = P.sum(dim=(0, 1, 2))
    hi = P[high].sum(dim=0)
    return torch.where(tot > 0, hi / torch.where(tot > 0, tot, torch.ones_like(tot)), torch.zeros_like(tot))


def select_channel_mask(field: "nh.Field", G: int = 64, cutoff: float = 0.25, threshold: float = 0.85,
                        apply: bool = True):
    """Computes the mask of the field's L * F channels; with ``apply`` installs it.
    Returns (mask float32 [L * F], high-frequency fraction per channel)."""
    cfg = field.cfg
    D = cfg.n_levels * cfg.n_feat
    dev = field.params.device
    h = torch.empty(G ** 3 * D, device=dev)
    nh.encode_points(field, torch.from_numpy(voxel_grid(G)).to(dev), h)
    frac = high_frequency_fraction(h.view(G ** 3, D), G, cutoff).cpu().numpy()
    mask = np.where(frac > threshold, 0.0, 1.0).astype(np.float32)
    if apply:
        field.set_channel_mask(mask)
    return mask, frac
