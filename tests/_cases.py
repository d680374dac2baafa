"""Shared builders for the parity tests: one seeded case is fed to both the CUDA
library and the CPU oracle (inputs only; the two share no arithmetic)."""
import dataclasses

import numpy as np

import oracle
import synthetic as S


def oracle_geom(g: S.GeometryConfig):
    tab, du, dv = oracle.view_table(g.n_views, g.angle0_rad, g.span_rad, g.dso_mm, g.dsd_mm,
                                    g.det_du_mm, g.det_dv_mm, g.vol_side_mm)
    return (tab, du, dv, g.det_nu, g.det_nv)


def hit_pixels(g: S.GeometryConfig, view: int):
    """Pixels whose ray meets the volume (oracle ray setup), for building batches."""
    tab, du, dv, nu, nv = oracle_geom(g)
    _, _, _, _, hit = oracle.ray_setup(tab, du, dv, nu, nv, view, np.arange(nu * nv))
    return np.nonzero(hit)[0]


def field_cfg(**kw):
    base = dict(n_levels=8, n_feat=2, log2_T=12, base_res=4, max_res=48, norm=S.NORM_LN,
                hidden_layers=2, width=32)
    base.update(kw)
    return S.FieldConfig(**base)


def batch(g: S.GeometryConfig, view: int, R: int, seed: int, n_miss: int = 0):
    rng = np.random.default_rng(seed)
    hits = hit_pixels(g, view)
    pix = rng.choice(hits, size=min(R, len(hits)), replace=R > len(hits)).astype(np.int32)
    if n_miss:
        miss = np.setdiff1d(np.arange(g.det_nu * g.det_nv), hits)
        pix = np.concatenate([pix, rng.choice(miss, size=n_miss)]).astype(np.int32)
    return pix


def rounded_tables(flat, cfg, precision):
    """The float32 parameter vector with its table part rounded the way the library's
    low-precision working copy stores it (round to nearest even)."""
    import torch
    out = np.array(flat, dtype=np.float32, copy=True)
    n = cfg.n_levels * cfg.T * cfg.n_feat
    if precision == S.PREC_BF16:
        out[:n] = torch.from_numpy(out[:n]).to(torch.bfloat16).float().numpy()
    elif precision == S.PREC_F16:
        out[:n] = torch.from_numpy(out[:n]).to(torch.float16).float().numpy()
    return out


# Seeded 16^3 sub-instance of the large configuration: the L16 F2 16..2048 field with
# T = 2^8 (level 0 dense, every other level hashed with forced collisions), one
# LayerNorm and the 4x32 MLP, on 4 views of an 8x8 detector.
C4_SUB = S.FieldConfig(n_levels=16, n_feat=2, log2_T=8, base_res=16, max_res=2048, norm=S.NORM_LN,
                       hidden_layers=4, width=32)
C4_SUB_GEOM = S.GeometryConfig(n_views=4, det_nu=8, det_nv=8)
C4_SUB_N = 16


def c4_subinstance(seed=11):
    """(oracle geometry, float64 params, pix, A_meas): measurements are the oracle
    projections (view 1) of a 16^3 shell phantom of the large workload's family, 6
    rays that meet the volume and one that misses."""
    geom = oracle_geom(C4_SUB_GEOM)
    vol, _ = S.phantom(S.WORKLOADS["large_bf16"], seed, D=16)
    proj = oracle.project(geom, vol, oversample=2)
    pix = batch(C4_SUB_GEOM, 1, 6, seed, n_miss=1)
    A_meas = proj[1].reshape(-1)[pix]
    flat = S.init_params(C4_SUB, seed, table_scale=0.5).astype(np.float64)
    return geom, flat, pix, A_meas


def replace(cfg, **kw):
    return dataclasses.replace(cfg, **kw)
