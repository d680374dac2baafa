"""FFT channel masking of the hash features (Sec. 2.3): argument marshalling only.

Some channels of the hash features carry noise rather than structure; the paper
tells them apart with a Fast Fourier Transform and masks them during training, but
gives no grid, statistic or threshold. The library's field_select_channel_mask
computes the reading documented in include/nhcbct.h: each channel of the hash
features (before normalization) sampled at the voxel centres of a G^3 grid, its
mean removed, the share of its 3-D power spectrum beyond |k| > cutoff cycles per
voxel; a channel whose share exceeds the threshold gets mask 0. White noise puts
about 0.93 of its power beyond a cutoff of 1/4, a smooth field almost none.

The selection is an occasional step between training steps, not part of the step
itself; the mask multiply inside the training kernels is.
"""
from __future__ import annotations

import numpy as np
import torch

from . import nhcbct as nh


def select_channel_mask(field: "nh.Field", G: int = 64, cutoff: float = 0.25, threshold: float = 0.85,
                        apply: bool = True, stream=None):
    """Computes the mask of the field's L * F channels on the GPU; with ``apply``
    installs it. Returns (mask float32 [L * F], high-frequency fraction per channel)
    as host arrays (the call synchronizes the stream to read them)."""
    cfg = field.cfg
    D = cfg.n_levels * cfg.n_feat
    dev = field.params.device
    ws = nh.workspace(nh.channel_mask_workspace_bytes(field, G), dev)
    frac = torch.empty(D, dtype=torch.float64, device=dev)
    mask = torch.empty(D, dtype=torch.float32, device=dev)
    nh.select_channel_mask(field, G, cutoff, threshold, apply, frac, mask, ws, stream)
    (stream if stream is not None else torch.cuda.current_stream()).synchronize()
    return mask.cpu().numpy().astype(np.float32), frac.cpu().numpy()
