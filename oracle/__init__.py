"""CPU oracle for the NeRF-CBCT training step (test infrastructure only).

A plain, slow, obviously-correct restatement of what the CUDA path computes,
written from the paper ("NeRF-based CBCT Reconstruction needs Normalization
and Initialization"): Beer-Lambert ray sum (Sec. 2.2, Eq. 1), the Normalized
Hash Encoder (Sec. 2.3), the voxel loss of Mapping Consistency Initialization
(Sec. 2.4, Eq. 2) and the pixel loss of sparse-view training (Sec. 2.5, Eq. 3),
optimized with Adam (Sec. 3.1).

Arithmetic is float64, except the sample-position / hash-index prefix, which is
a sequence of individually rounded float32 operations so that positions and
corner indices can be compared bit for bit with the GPU.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg
may import this package. It shares no code with the CUDA library and never
imports it; both sides receive the same seeded inputs from ``synthetic``.

Parity status: every function here is pinned by a ``-m "not gpu"`` test against
a closed form, a library routine, brute force or finite differences, except the
transfer *gain* of Mapping Consistency Initialization, which has no closed form
(parity unpinned; it is measured against random initialization instead). The FFT
channel mask (mask.py) is pinned on pure tones, white noise and planted fields;
the paper gives no grid, statistic or threshold, so those are a stated reading.
The 3-D SSIM (ssim.py) is pinned on identical and constant volumes, on brute force
over one window, and on a library filter.
"""
from .geometry import view_table, ray_setup, sample_points, voxel_centres_f32, splitmix64, stratum_offsets
from .encoding import level_resolutions, corners, encode, encode_backward
from .field import (unflatten, flatten, normalize_forward, normalize_backward,
                    mlp_forward, mlp_backward, field_forward, field_backward)
from .train import (render, loss_and_grad, render_forward, render_backward, adam_step,
                    train_step, fit_points_step, query_points, query_volume, AdamState)
from .project import project
from .mask import radial_frequency, high_frequency_fraction, mask_from_fraction, channel_mask
from .ssim import gaussian_window, ssim_map, ssim

__all__ = [
    "view_table", "ray_setup", "sample_points", "voxel_centres_f32", "splitmix64", "stratum_offsets",
    "level_resolutions", "corners", "encode", "encode_backward",
    "unflatten", "flatten", "normalize_forward", "normalize_backward",
    "mlp_forward", "mlp_backward", "field_forward", "field_backward",
    "render", "loss_and_grad", "render_forward", "render_backward", "adam_step",
    "train_step", "fit_points_step", "query_points", "query_volume", "AdamState",
    "project", "radial_frequency", "high_frequency_fraction", "mask_from_fraction", "channel_mask",
    "gaussian_window", "ssim_map", "ssim",
]
