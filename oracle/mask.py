"""FFT channel masking of the hash features (Sec. 2.3), test infrastructure.

The paper says only that some channels of the hash features carry meaningless
noise and that a Fast Fourier Transform tells them apart, so that they can be
masked during training. It gives no grid, statistic or threshold. The reading
restated here:

- every channel of the hash features h (before normalization) is sampled at the
  voxel centres (k + 1/2) / G of a G^3 grid over the volume, the grid on which the
  reconstruction is read out;
- each channel's mean is removed and its 3-D power spectrum |FFT|^2 taken;
- the channel's high-frequency fraction is the share of that power at radial
  frequencies |k| > cutoff (cycles per voxel, |k| in [0, sqrt(3)/2]);
- a channel whose fraction exceeds the threshold is noise-like and gets mask 0;
  every other channel (including one with no variance) keeps mask 1.

White noise puts (number of bins beyond the cutoff) / (G^3 - 1) of its power
there (0.93 at cutoff 1/4), a smooth channel almost none.
"""
import numpy as np

from .encoding import encode, level_resolutions
from .field import unflatten


def radial_frequency(G):
    """|k| (cycles per voxel) of every bin of a G^3 FFT, shape (G, G, G)."""
    f = np.fft.fftfreq(G)
    kz, ky, kx = np.meshgrid(f, f, f, indexing="ij")
    return np.sqrt(kx * kx + ky * ky + kz * kz)


def high_frequency_fraction(h, G, cutoff):
    """Per channel of h (G^3, C) in [z][y][x] order: power share at |k| > cutoff."""
    h = np.asarray(h, dtype=np.float64).reshape(G, G, G, -1)
    h = h - h.mean(axis=(0, 1, 2), keepdims=True)
    P = np.abs(np.fft.fftn(h, axes=(0, 1, 2))) ** 2
    high = radial_frequency(G) > cutoff
    tot = P.sum(axis=(0, 1, 2))
    hi = P[high].sum(axis=0)
    return np.where(tot > 0, hi / np.where(tot > 0, tot, 1.0), 0.0)


def mask_from_fraction(frac, threshold):
    return np.where(np.asarray(frac) > threshold, 0.0, 1.0)


def voxel_grid(G):
    """(G^3, 3) float32 voxel centres (k + 1/2) / G, flattened [z][y][x]."""
    c = (np.arange(G, dtype=np.float32) + np.float32(0.5)) / np.float32(G)
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=-1).astype(np.float32)


def channel_mask(flat, cfg, G=64, cutoff=0.25, threshold=0.85):
    """(mask, fraction) of the field's L * F hash-feature channels."""
    p = unflatten(np.asarray(flat, dtype=np.float64), cfg)
    res = level_resolutions(cfg.n_levels, cfg.base_res, cfg.max_res)
    h = encode(voxel_grid(G), p["tables"], res, cfg.T)
    frac = high_frequency_fraction(h, G, cutoff)
    return mask_from_fraction(frac, threshold), frac
