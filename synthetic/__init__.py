"""Seeded synthetic inputs for the NeRF-CBCT training step.

This module makes the data that both the CUDA path and the CPU oracle consume:
ellipsoid phantoms, per-step ray picks, initial parameter vectors, Poisson
measurement noise and the named workload shapes. It holds none of the method's
arithmetic (no sampling, hashing, normalization, MLP, ray sum or loss), so the
two implementations under test share inputs only, never computation.

The public CT datasets the paper evaluates on (Sec. 3.1: Covid-19 chest,
Pancreas_CT, HAN_seg, the R2-Gaussian cases) are not available; seeded
ellipsoid phantoms with values in [0, 1] stand in for them, projected with the
same cone-beam geometry family (50 views over 360 degrees, source-to-origin
1000 mm, source-to-detector 1500 mm).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "GeometryConfig", "FieldConfig", "Workload", "WORKLOADS",
    "EllipsoidSet", "random_ellipsoids", "paint_ellipsoids", "smooth_texture",
    "phantom", "param_layout", "init_params", "pick_rays", "poisson_measure",
    "random_points",
]

NORM_NONE, NORM_LN, NORM_LN_PER_LEVEL = 0, 1, 2
PREC_F32, PREC_BF16, PREC_F16 = 0, 1, 2
LOSS_MSE, LOSS_L1 = 0, 1


@dataclasses.dataclass(frozen=True)
class GeometryConfig:
    """Cone-beam scanner: circular source orbit about the volume's z axis."""
    n_views: int = 50
    angle0_rad: float = 0.0
    span_rad: float = 2.0 * math.pi
    dso_mm: float = 1000.0
    dsd_mm: float = 1500.0
    det_nu: int = 64
    det_nv: int = 64
    det_side_mm: float = 700.0     # detector is square; pitch = side / n
    vol_side_mm: float = 256.0     # cube centred at the origin

    @property
    def det_du_mm(self) -> float:
        return self.det_side_mm / self.det_nu

    @property
    def det_dv_mm(self) -> float:
        return self.det_side_mm / self.det_nv


@dataclasses.dataclass(frozen=True)
class FieldConfig:
    """Hash-grid + normalization + MLP field and its optimizer settings."""
    n_levels: int = 8
    n_feat: int = 2
    log2_T: int = 14
    base_res: int = 16
    max_res: int = 64
    norm: int = NORM_LN
    ln_eps: float = 1e-5
    hidden_layers: int = 2
    width: int = 32
    precision: int = PREC_F32
    loss: int = LOSS_MSE
    lr: float = 1e-3
    beta1: float = 0.9
    beta2: float = 0.999
    adam_eps: float = 1e-8
    loss_scale_init: float = 1.0
    growth_interval: int = 0       # 0: static loss scale

    @property
    def d_in(self) -> int:
        return self.n_levels * self.n_feat

    @property
    def T(self) -> int:
        return 1 << self.log2_T


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    vol_D: int
    n_ellipsoids: int
    texture: bool
    shells: bool
    geometry: GeometryConfig
    field: FieldConfig
    n_rays: int
    n_samples: int
    steps: int
    I0: float = 1e5

    @property
    def samples_per_step(self) -> int:
        return self.n_rays * self.n_samples


_G50_64 = GeometryConfig(det_nu=64, det_nv=64)
_G50_256 = GeometryConfig(det_nu=256, det_nv=256)
_G100_512 = GeometryConfig(n_views=100, det_nu=512, det_nv=512)

_F_TINY = FieldConfig(n_levels=8, n_feat=2, log2_T=14, base_res=16, max_res=64,
                      norm=NORM_LN_PER_LEVEL, hidden_layers=2, width=32)
_F_PAPER = FieldConfig(n_levels=16, n_feat=2, log2_T=19, base_res=16, max_res=2048,
                       norm=NORM_LN, hidden_layers=4, width=32)
_F_LARGE = dataclasses.replace(_F_PAPER, log2_T=21, precision=PREC_BF16)

WORKLOADS = {
    # 64^3, 5 ellipsoids, 64x64 detector, L8 F2 T2^14, per-level normalization, 2x32 MLP
    "tiny_fp32": Workload("tiny_fp32", 64, 5, False, False, _G50_64, _F_TINY, 1024, 64, 100),
    # 128^3 textured, 256^2 detector, L16 F2 T2^19, layer norm, 4x32 MLP, 2048 rays x 192 samples
    "paper_fp32": Workload("paper_fp32", 128, 10, True, False, _G50_256, _F_PAPER, 2048, 192, 3000),
    # the tiny workload with BF16 tables and tensor-core MLP
    "tiny_bf16": Workload("tiny_bf16", 64, 5, False, False, _G50_64,
                          dataclasses.replace(_F_TINY, precision=PREC_BF16), 1024, 64, 100),
    "tiny_f16": Workload("tiny_f16", 64, 5, False, False, _G50_64,
                         dataclasses.replace(_F_TINY, precision=PREC_F16, loss_scale_init=1024.0,
                                             growth_interval=200), 1024, 64, 100),
    # the paper-scale shape in mixed precision (for the mixed-vs-FP32 comparison)
    "paper_bf16": Workload("paper_bf16", 128, 10, True, False, _G50_256,
                           dataclasses.replace(_F_PAPER, precision=PREC_BF16), 2048, 192, 3000),
    # the paper's own step shape (Sec. 3.1): one view, 1024 rays x 320 samples, the L1
    # pixel loss of Eq. 3, on the paper-scale field and scan
    "paper320_fp32": Workload("paper320_fp32", 128, 10, True, False, _G50_256,
                              dataclasses.replace(_F_PAPER, loss=LOSS_L1), 1024, 320, 3000),
    "paper320_bf16": Workload("paper320_bf16", 128, 10, True, False, _G50_256,
                              dataclasses.replace(_F_PAPER, loss=LOSS_L1, precision=PREC_BF16), 1024, 320, 3000),
    # 256^3 with bone-like shells, 100 views of 512^2, T=2^21, 8192 rays x 256 samples, BF16
    "large_bf16": Workload("large_bf16", 256, 20, False, True, _G100_512, _F_LARGE, 8192, 256, 3000),
}


# ----------------------------------------------------------------------------------------
# Phantoms
# ----------------------------------------------------------------------------------------
@dataclasses.dataclass
class EllipsoidSet:
    """Ellipsoids in volume units (cube side 1, centred at the origin), painted in order."""
    centres: np.ndarray    # (K, 3)
    axes: np.ndarray       # (K, 3) semi-axes
    rot: np.ndarray        # (K, 3, 3) columns are the principal directions (local = (x - c) @ rot)
    values: np.ndarray     # (K,)


def _haar_rotation(rng: np.random.Generator) -> np.ndarray:
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def random_ellipsoids(K: int, seed: int, shells: bool = False) -> EllipsoidSet:
    """K random ellipsoids: centres U[-0.35,0.35]^3, semi-axes U[0.04,0.25],
    Haar-random orientation, value U[0,1]. With ``shells``, every ellipsoid
    becomes a bone-like shell: an outer ellipsoid of value U[0.8,1.0] followed by
    an inner copy scaled by U[0.85,0.92] that restores the base value."""
    rng = np.random.default_rng(seed)
    c, a, r, v = [], [], [], []
    for _ in range(K):
        ck = rng.uniform(-0.35, 0.35, size=3)
        ak = rng.uniform(0.04, 0.25, size=3)
        rk = _haar_rotation(rng)
        vk = rng.uniform(0.0, 1.0)
        if shells:
            c.append(ck); a.append(ak); r.append(rk); v.append(rng.uniform(0.8, 1.0))
            ak = ak * rng.uniform(0.85, 0.92)
        c.append(ck); a.append(ak); r.append(rk); v.append(vk)
    return EllipsoidSet(np.array(c), np.array(a), np.array(r), np.array(v))


def voxel_centres(D: int) -> np.ndarray:
    """Voxel-centre coordinates in centred volume units, shape (D, D, D, 3), [z][y][x]."""
    g = (np.arange(D) + 0.5) / D - 0.5
    z, y, x = np.meshgrid(g, g, g, indexing="ij")
    return np.stack([x, y, z], axis=-1)


def paint_ellipsoids(E: EllipsoidSet, D: int) -> np.ndarray:
    """Piecewise-constant volume (D^3, [z][y][x], float64): later ellipsoids overwrite.
    Each ellipsoid is tested only on the voxels of the cube that holds its bounding
    sphere (radius = its largest semi-axis, plus one voxel), since no voxel outside
    that sphere can lie inside it."""
    g = (np.arange(D) + 0.5) / D - 0.5
    vol = np.zeros((D, D, D))
    for k in range(len(E.values)):
        c, rot, ax = E.centres[k], E.rot[k], E.axes[k]
        rad = float(ax.max()) + 1.0 / D
        lo = np.searchsorted(g, c - rad, side="left")
        hi = np.searchsorted(g, c + rad, side="right")
        if np.any(hi <= lo):
            continue
        z, y, x = np.meshgrid(g[lo[2]:hi[2]] - c[2], g[lo[1]:hi[1]] - c[1], g[lo[0]:hi[0]] - c[0], indexing="ij")
        q = 0.0
        for j in range(3):                                  # coordinates along principal axis j
            local = x * rot[0, j] + y * rot[1, j] + z * rot[2, j]
            q = q + (local / ax[j]) ** 2
        sub = vol[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]]
        sub[q <= 1.0] = E.values[k]
    return vol


def smooth_texture(D: int, seed: int, n_bumps: int = 8) -> np.ndarray:
    """1 + 0.3 * sum of Gaussian bumps (amplitude U[-1,1], width U[0.05,0.15])."""
    rng = np.random.default_rng(seed)
    X = voxel_centres(D)
    tex = np.ones((D, D, D))
    for _ in range(n_bumps):
        c = rng.uniform(-0.5, 0.5, size=3)
        s = rng.uniform(0.05, 0.15)
        amp = rng.uniform(-1.0, 1.0)
        tex += 0.3 * amp * np.exp(-np.sum((X - c) ** 2, axis=-1) / (2 * s * s))
    return tex


def phantom(w: Workload, seed: int, D: int | None = None):
    """Volume of workload ``w`` (values clamped to [0, 1]) and its ellipsoids."""
    D = w.vol_D if D is None else D
    E = random_ellipsoids(w.n_ellipsoids, seed, shells=w.shells)
    vol = paint_ellipsoids(E, D)
    if w.texture:
        vol = np.clip(vol * smooth_texture(D, seed + 7919), 0.0, 1.0)
    return vol, E


# ----------------------------------------------------------------------------------------
# Parameters and batches
# ----------------------------------------------------------------------------------------
def param_layout(f: FieldConfig) -> dict:
    """Offsets (in floats) of each parameter group in the flat parameter vector:
    tables [L][T][F], gamma [D], beta [D], then W_k [out][in] and b_k [out] per layer."""
    L, F, T, D, W, H = f.n_levels, f.n_feat, f.T, f.d_in, f.width, f.hidden_layers
    off = {"tables": (0, L * T * F)}
    o = L * T * F
    off["gamma"] = (o, D); o += D
    off["beta"] = (o, D); o += D
    dims = [D] + [W] * H + [1]
    for k in range(H + 1):
        off[f"W{k}"] = (o, dims[k + 1] * dims[k]); o += dims[k + 1] * dims[k]
        off[f"b{k}"] = (o, dims[k + 1]); o += dims[k + 1]
    off["_total"] = (0, o)
    off["_dims"] = dims
    return off


def init_params(f: FieldConfig, seed: int, table_scale: float = 1e-4) -> np.ndarray:
    """Flat float32 parameters: tables U(-1e-4, 1e-4), gamma 1, beta 0, and
    W_k, b_k ~ U(-1/sqrt(fan_in), 1/sqrt(fan_in)) (PyTorch's Linear default)."""
    rng = np.random.default_rng(seed)
    lay = param_layout(f)
    p = np.zeros(lay["_total"][1], dtype=np.float32)
    o, n = lay["tables"]
    p[o:o + n] = rng.uniform(-table_scale, table_scale, size=n)
    o, n = lay["gamma"]
    p[o:o + n] = 1.0
    dims = lay["_dims"]
    for k in range(len(dims) - 1):
        bound = 1.0 / math.sqrt(dims[k])
        for name in (f"W{k}", f"b{k}"):
            o, n = lay[name]
            p[o:o + n] = rng.uniform(-bound, bound, size=n)
    return p


def pick_rays(rng: np.random.Generator, n_views: int, candidates, R: int):
    """One view per batch (Sec. 3.1: batch size of views is 1) and R distinct pixels of it.

    ``candidates[v]`` lists the pixel ids (row * nu + col) of view v that a batch may
    use, normally those whose ray meets the volume, so that every ray carries samples.
    The drawn pixels come back in ascending id (detector raster order). The loss and
    the gradients do not depend on the order beyond float rounding, but rays that sit
    next to each other in the batch run side by side on the GPU, and neighbouring rays
    touch neighbouring table entries, which the L2 then serves.
    """
    view = int(rng.integers(0, n_views))
    cand = np.asarray(candidates[view])
    sel = rng.choice(len(cand), size=R, replace=(R > len(cand)))
    return view, np.sort(cand[sel]).astype(np.int32)


def poisson_measure(A_clean: np.ndarray, I0: float, seed: int) -> np.ndarray:
    """Measured projections: I ~ Poisson(I0 exp(-A)), A_meas = -ln(max(I, 1) / I0)."""
    rng = np.random.default_rng(seed)
    I = rng.poisson(I0 * np.exp(-np.asarray(A_clean, dtype=np.float64)))
    return (-np.log(np.maximum(I, 1) / I0)).astype(np.float32)


def random_points(rng: np.random.Generator, D: int, P: int):
    """P random voxel indices of a D^3 grid, as (flat index, voxel-centre xyz in [0,1]^3 f32)."""
    idx = rng.integers(0, D ** 3, size=P)
    z, rem = np.divmod(idx, D * D)
    y, x = np.divmod(rem, D)
    xyz = (np.stack([x, y, z], axis=-1) + 0.5) / D
    return idx, xyz.astype(np.float32)
