"""Shared builders for the parity tests: one seeded case is fed to both the CUDA
library and the CPU oracle (inputs only; the two share no arithmetic), and the
tolerance helpers of the FP32 gradient comparison."""
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


def kink_free_rays(cache, n_rays, rel=4e-6):
    """Indices of the batch's rays none of whose samples has a hidden ReLU unit
    within float32 rounding of its kink (|z| <= rel * (sum_i |W_ji a_i| + |b_j|), the
    criterion of table_kink_allowance). At such a unit either branch is a correct
    float32 result; a batch without them has one correct gradient, which FP32
    implementations must reach within rounding in every parameter group."""
    p, fc, hit, delta, N = cache
    keep = np.ones(n_rays, dtype=bool)
    if fc is None:
        return np.nonzero(keep)[0]
    x, res, T, mask, ncache, mu, acts, zs = fc
    Ws, bs = p["W"], p["b"]
    amb = np.zeros(len(mu), dtype=bool)
    for k in range(len(Ws) - 1):
        scale = np.abs(acts[k]) @ np.abs(Ws[k]).T + np.abs(bs[k])
        amb |= np.any(np.abs(zs[k]) <= rel * scale, axis=1)
    hit_rays = np.nonzero(hit)[0]
    keep[np.unique(hit_rays[np.nonzero(amb)[0] // N])] = False
    return np.nonzero(keep)[0]


def table_kink_allowance(cache, dLdA, cfg, rel=4e-6):
    """Elementwise bound on how far a float32 implementation's hash-table gradient
    may lie from the oracle's because a ReLU unit whose pre-activation is within
    float32 rounding of zero took the other branch. The ReLU derivative jumps at 0,
    so for such a unit both branches follow from the same arithmetic to within
    rounding, and either is a correct result. A flipped unit j of layer k adds or
    removes the gradient path through it: dL/da_{k+1,j} W_k[j, :] at the layer's
    input, carried down to the hash tables.

    A hidden unit is ambiguous when |z| <= rel * (sum_i |W_ji a_i| + |b_j|): the
    float32 error bound of a 32-term dot product is about 32 u = 1.9e-6 of that sum
    (u = 2^-24), and rel = 4e-6 leaves room for the error its inputs carry in. The
    bound sums, over the ambiguous units of each sample, the magnitude of that path
    (|dL/da_{k+1,j}| |W_k[j, :]|, then |W|, |gamma|, |hhat| and the LayerNorm
    backward on magnitudes, with ambiguous units passing gradient), scattered with
    the trilinear weights. It is returned as a flat vector shaped like the gradient,
    zero outside the tables; entries no ambiguous sample reaches get none."""
    from oracle import field as OF
    from oracle.encoding import encode_backward
    p, fc, hit, delta, N = cache
    n = OF.flatten(p).size
    if fc is None:
        return np.zeros(n)
    x, res, T, mask, ncache, mu, acts, zs = fc
    Ws, bs = p["W"], p["b"]
    H = len(Ws) - 1
    amb = []
    for k in range(H):
        scale = np.abs(acts[k]) @ np.abs(Ws[k]).T + np.abs(bs[k])
        amb.append(np.abs(zs[k]) <= rel * scale)
    S = np.nonzero(np.any(np.stack([a.any(axis=1) for a in amb]), axis=0))[0]
    out = np.zeros(n)
    if len(S) == 0:
        return out
    dmu = np.repeat(np.asarray(dLdA, dtype=np.float64)[hit] * delta[hit].astype(np.float64), N)[S]
    # dL/da_{k+1} (the gradient arriving at each hidden unit's output) under the
    # oracle's branches
    dz = (dmu * mu[S] * (1.0 - mu[S]))[:, None]
    da_out = [None] * H
    for k in range(H, 0, -1):
        da = dz @ Ws[k]
        da_out[k - 1] = da
        dz = da * (zs[k - 1][S] > 0.0)
    # t bounds the change of dL/da at the input of layer k, from the flips at or
    # above layer k, carried down layer by layer
    t = np.zeros((len(S), Ws[H].shape[1]))
    for k in range(H - 1, -1, -1):
        t = (t * ((zs[k][S] > 0.0) | amb[k][S]) + np.abs(da_out[k]) * amb[k][S]) @ np.abs(Ws[k])
    G = 1 if cfg.norm == 1 else (cfg.n_levels if cfg.norm == 2 else 0)
    D = t.shape[1]
    gch = t * np.abs(mask)
    if G == 0:
        dh = gch
    else:
        hhat, rstd = ncache
        dhh = (gch * np.abs(p["gamma"])).reshape(len(S), G, D // G)
        hg = np.abs(hhat[S]).reshape(len(S), G, D // G)
        dh = (rstd[S][:, :, None] * (dhh + dhh.mean(axis=-1, keepdims=True)
                                      + hg * (dhh * hg).mean(axis=-1, keepdims=True))).reshape(len(S), D)
    tables = encode_backward(x[S], dh, res, T, cfg.n_feat)
    out[: tables.size] = tables.ravel()
    return out


def fp32_gradient_errors(g, g_ref, cfg, cache, dLdA, tol=1e-3):
    """Groups whose float32 gradient misses the oracle's, for the FP32 paths.

    Dense groups (gamma, beta, W_k, b_k): every entry within tol of the group's
    largest entry. Hash tables: the entries that no ReLU-ambiguous sample reaches
    (see table_kink_allowance) within tol of the largest table entry, and their
    error norm within tol of the table gradient's norm; every entry within tol of
    the largest entry plus the kink allowance. Returns {group: errors} of the
    failing groups, and prints every group's errors."""
    lay = S.param_layout(cfg)
    allow = table_kink_allowance(cache, dLdA, cfg)
    names = ("tables", "gamma", "beta") + tuple(f"{p}{k}" for k in range(cfg.hidden_layers + 1) for p in ("W", "b"))
    bad, report = {}, {}
    for name in names:
        o, n = lay[name]
        a, b = g[o:o + n].astype(np.float64), g_ref[o:o + n]
        scale = np.abs(b).max()
        d = np.abs(a - b)
        if scale == 0:
            if d.max() > 0:
                bad[name] = (np.inf, np.inf)
            continue
        err = (d.max() / scale, np.linalg.norm(a - b) / np.linalg.norm(b))
        if name == "tables":
            al = allow[o:o + n]
            strict = al == 0
            err = (d[strict].max() / scale, float(np.linalg.norm(d[strict]) / np.linalg.norm(b)),
                   float(np.max(d - al) / scale), float(np.mean(~strict)))
            ok = err[0] <= tol and err[1] <= tol and err[2] <= tol
        else:
            ok = err[0] <= tol
        report[name] = tuple(f"{e:.2e}" for e in err)
        if not ok:
            bad[name] = err
    print(report)
    return bad
