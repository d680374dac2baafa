"""3-D structural similarity, test infrastructure.

The paper reports SSIM beside PSNR (Sec. 3.2, and the view sweep and ablation of
Fig. 7 and 8). It cites Wang, Bovik, Sheikh and Simoncelli, "Image quality
assessment: from error visibility to structural similarity" (IEEE TIP 2004), and
gives no settings. The reading restated here keeps that paper's settings and
takes its windows from 2-D to 3-D:
- the window is a Gaussian of standard deviation 1.5 voxels, 11 voxels wide on
  each axis, normalised to sum 1: w(i, j, k) = g(i) g(j) g(k), g(t) proportional
  to exp(-t^2 / (2 * 1.5^2)) for t = -5..5;
- at each window position that lies wholly inside the volume ((D - 10)^3 "valid"
  positions) the window gives the weighted means mu_x, mu_y, the weighted
  variances sigma_x^2 = sum w (x - mu_x)^2, sigma_y^2 and the covariance
  sigma_xy = sum w (x - mu_x)(y - mu_y);
- the local index there is
  (2 mu_x mu_y + C1)(2 sigma_xy + C2) / ((mu_x^2 + mu_y^2 + C1)(sigma_x^2 + sigma_y^2 + C2)),
  with C1 = (K1 L)^2, C2 = (K2 L)^2, K1 = 0.01, K2 = 0.03 and L the data range
  (1 for volumes in [0, 1]);
- the score is the mean of the local index over the valid positions.

Everything is FP64, and each window is summed directly over its 11^3 voxels,
one output plane at a time, so that the code reads as the definition.
"""
import numpy as np

RADIUS = 5          # window half-width: 11 voxels per axis
SIGMA = 1.5         # Gaussian standard deviation, voxels
K1, K2 = 0.01, 0.03


def gaussian_window(radius=RADIUS, sigma=SIGMA):
    """1-D weights g(t), t = -radius..radius, summing to 1 (FP64)."""
    t = np.arange(-radius, radius + 1, dtype=np.float64)
    g = np.exp(-(t * t) / (2.0 * sigma * sigma))
    return g / g.sum()


def ssim_map(x, y, data_range=1.0, radius=RADIUS, sigma=SIGMA):
    """Local SSIM index at every valid window position of two (D, D, D) volumes in
    [z][y][x] order; returns an (M, M, M) FP64 array, M = D - 2 * radius."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    D = x.shape[0]
    assert x.shape == (D, D, D) and y.shape == (D, D, D) and D > 2 * radius
    W = 2 * radius + 1
    M = D - 2 * radius
    g = gaussian_window(radius, sigma)
    w = g[:, None, None] * g[None, :, None] * g[None, None, :]   # w[dz, dy, dx]
    c1 = (K1 * data_range) ** 2
    c2 = (K2 * data_range) ** 2
    wx = np.lib.stride_tricks.sliding_window_view(x, (W, W, W))   # (M, M, M, W, W, W)
    wy = np.lib.stride_tricks.sliding_window_view(y, (W, W, W))
    out = np.empty((M, M, M))
    for z in range(M):
        bx, by = wx[z], wy[z]                                     # (M, M, W, W, W)
        mx = np.einsum("abijk,ijk->ab", bx, w)
        my = np.einsum("abijk,ijk->ab", by, w)
        dx = bx - mx[:, :, None, None, None]
        dy = by - my[:, :, None, None, None]
        vx = np.einsum("abijk,ijk->ab", dx * dx, w)
        vy = np.einsum("abijk,ijk->ab", dy * dy, w)
        cxy = np.einsum("abijk,ijk->ab", dx * dy, w)
        out[z] = ((2.0 * mx * my + c1) * (2.0 * cxy + c2)) / ((mx * mx + my * my + c1) * (vx + vy + c2))
    return out


def ssim(x, y, data_range=1.0):
    """Mean SSIM of two (D, D, D) volumes (the score reported beside PSNR)."""
    return float(ssim_map(x, y, data_range).mean())
