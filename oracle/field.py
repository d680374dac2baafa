"""The field M(x, y, z): hash encoding -> Normalized Hash Encoder -> MLP (oracle).

Test infrastructure: only the tests, the smoke check and the benchmark's CPU legs
use it.

Sec. 2.3 places a Layer Normalization between the hash encoder and the neural
network so that the features keep one global mean and variance, and masks
feature channels found to carry noise. The equation the text announces is
missing from it, and the text describes LN both as per-point and as
batch-wide. The reading used here is PyTorch's LayerNorm applied to each
point's own feature vector (biased variance, eps, learnable gamma and beta), in
one of three modes:

* ``norm == 0`` (none):   y = h * m;
* ``norm == 1`` (LN):     one group of all L*F features;
* ``norm == 2`` (per level): L groups of F features each;

  y = (gamma * (h - mean_g) / sqrt(var_g + eps) + beta) * m,

with m the channel mask (ones unless set). The MLP ("neural network", Sec. 1)
maps y through H hidden Linear+ReLU layers of width W and a Linear layer to
one output, and sigmoid gives the attenuation mu. Linear layers carry a bias.

Flat parameter layout (shared with the CUDA library as a data format only):
tables [L][T][F], gamma [D], beta [D], then W_k [out][in] and b_k [out] for
k = 0..H, with D = L * F.
"""
from __future__ import annotations

import numpy as np

from .encoding import level_resolutions, encode, encode_backward


def _dims(cfg):
    D = cfg.n_levels * cfg.n_feat
    return [D] + [cfg.width] * cfg.hidden_layers + [1]


def unflatten(flat, cfg):
    """Flat parameter vector -> dict of float64 arrays."""
    flat = np.asarray(flat, dtype=np.float64)
    L, F, T = cfg.n_levels, cfg.n_feat, 1 << cfg.log2_T
    dims = _dims(cfg)
    D = dims[0]
    o = 0
    p = {"tables": flat[o:o + L * T * F].reshape(L, T, F)}
    o += L * T * F
    p["gamma"] = flat[o:o + D]; o += D
    p["beta"] = flat[o:o + D]; o += D
    p["W"], p["b"] = [], []
    for k in range(len(dims) - 1):
        n = dims[k + 1] * dims[k]
        p["W"].append(flat[o:o + n].reshape(dims[k + 1], dims[k])); o += n
        p["b"].append(flat[o:o + dims[k + 1]]); o += dims[k + 1]
    assert o == flat.size, (o, flat.size)
    return p


def flatten(p):
    parts = [p["tables"].ravel(), p["gamma"], p["beta"]]
    for W, b in zip(p["W"], p["b"]):
        parts += [W.ravel(), b]
    return np.concatenate(parts).astype(np.float64)


def _groups(cfg):
    D = cfg.n_levels * cfg.n_feat
    return 1 if cfg.norm == 1 else (cfg.n_levels if cfg.norm == 2 else 0), D


def normalize_forward(h, gamma, beta, mask, cfg):
    """Normalized Hash Encoder (Sec. 2.3). Returns y and a cache for the backward."""
    G, D = _groups(cfg)
    if G == 0:
        return h * mask, None
    P = h.shape[0]
    hg = h.reshape(P, G, D // G)
    mean = hg.mean(axis=-1, keepdims=True)
    var = ((hg - mean) ** 2).mean(axis=-1, keepdims=True)
    rstd = 1.0 / np.sqrt(var + cfg.ln_eps)
    hhat = ((hg - mean) * rstd).reshape(P, D)
    y = (gamma * hhat + beta) * mask
    return y, (hhat, rstd.reshape(P, G))


def normalize_backward(dy, cache, gamma, mask, cfg):
    """Adjoint of ``normalize_forward``: returns dh, dgamma, dbeta."""
    G, D = _groups(cfg)
    if G == 0:
        return dy * mask, np.zeros(D), np.zeros(D)
    hhat, rstd = cache
    P = dy.shape[0]
    g = dy * mask
    dgamma = np.sum(g * hhat, axis=0)
    dbeta = np.sum(g, axis=0)
    dhhat = (g * gamma).reshape(P, G, D // G)
    hh = hhat.reshape(P, G, D // G)
    dh = rstd[:, :, None] * (dhhat - dhhat.mean(axis=-1, keepdims=True)
                             - hh * (dhhat * hh).mean(axis=-1, keepdims=True))
    return dh.reshape(P, D), dgamma, dbeta


def mlp_forward(y, Ws, bs):
    """ReLU MLP with sigmoid output. Returns mu (P,), layer inputs and pre-activations."""
    acts, zs = [y], []
    a = y
    for k, (W, b) in enumerate(zip(Ws, bs)):
        z = a @ W.T + b
        zs.append(z)
        if k < len(Ws) - 1:
            a = np.maximum(z, 0.0)
            acts.append(a)
    mu = 1.0 / (1.0 + np.exp(-zs[-1][:, 0]))
    return mu, acts, zs


def mlp_backward(dmu, mu, acts, zs, Ws):
    """Chain rule through the MLP (ReLU derivative 0 at 0). Returns dy, dWs, dbs."""
    dz = (dmu * mu * (1.0 - mu))[:, None]
    dWs, dbs = [None] * len(Ws), [None] * len(Ws)
    for k in range(len(Ws) - 1, -1, -1):
        dWs[k] = dz.T @ acts[k]
        dbs[k] = dz.sum(axis=0)
        da = dz @ Ws[k]
        if k > 0:
            dz = da * (zs[k - 1] > 0.0)
    return da, dWs, dbs


def field_forward(p, x, cfg, mask=None):
    """mu = M(x) at points x (P, 3) float32 in [0,1]^3. Returns (mu, cache)."""
    D = cfg.n_levels * cfg.n_feat
    mask = np.ones(D) if mask is None else np.asarray(mask, dtype=np.float64)
    res = level_resolutions(cfg.n_levels, cfg.base_res, cfg.max_res)
    T = 1 << cfg.log2_T
    h = encode(x, p["tables"], res, T)
    y, ncache = normalize_forward(h, p["gamma"], p["beta"], mask, cfg)
    mu, acts, zs = mlp_forward(y, p["W"], p["b"])
    return mu, (x, res, T, mask, ncache, mu, acts, zs)


def field_backward(p, cache, dmu, cfg):
    """Gradients (dict shaped like ``p``) of sum_i dmu_i * mu_i."""
    x, res, T, mask, ncache, mu, acts, zs = cache
    dy, dWs, dbs = mlp_backward(dmu, mu, acts, zs, p["W"])
    dh, dgamma, dbeta = normalize_backward(dy, ncache, p["gamma"], mask, cfg)
    dT = encode_backward(x, dh, res, T, cfg.n_feat)
    return {"tables": dT, "gamma": dgamma, "beta": dbeta, "W": dWs, "b": dbs}
