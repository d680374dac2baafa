"""Writes the stored expected values of tests/golden/: the CPU oracle's result for one
small seeded training step (Sec. 2.5, Eq. 1, Eq. 3, Sec. 3.1), so that later changes
to the oracle or the library are checked against a fixed record. It calls only the
oracle and the seeded input generators; run it from the repository root:

    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synthetic as S  # noqa: E402

GEOM = S.GeometryConfig(n_views=6, det_nu=24, det_nv=20)
FIELD = S.FieldConfig(n_levels=8, n_feat=2, log2_T=10, base_res=4, max_res=96, norm=S.NORM_LN,
                      hidden_layers=2, width=32)
VIEW, N, N_RAYS, SEED = 2, 40, 24, 7


def case():
    """(oracle geometry, float64 params, pix, a_meas) of the stored step."""
    tab, du, dv = oracle.view_table(GEOM.n_views, GEOM.angle0_rad, GEOM.span_rad, GEOM.dso_mm, GEOM.dsd_mm,
                                    GEOM.det_du_mm, GEOM.det_dv_mm, GEOM.vol_side_mm)
    geom = (tab, du, dv, GEOM.det_nu, GEOM.det_nv)
    _, _, _, _, hit = oracle.ray_setup(tab, du, dv, GEOM.det_nu, GEOM.det_nv, VIEW,
                                       np.arange(GEOM.det_nu * GEOM.det_nv))
    rng = np.random.default_rng(SEED)
    pix = np.sort(rng.choice(np.nonzero(hit)[0], size=N_RAYS, replace=False)).astype(np.int32)
    a_meas = rng.uniform(0.0, 0.6, size=N_RAYS).astype(np.float32)
    flat = S.init_params(FIELD, SEED, table_scale=0.5).astype(np.float64)
    return geom, flat, pix, a_meas


def expected():
    geom, flat, pix, a_meas = case()
    A, cache = oracle.render_forward(flat, FIELD, geom, VIEW, pix, N)
    loss, dLdA = oracle.loss_and_grad(A, a_meas, S.LOSS_MSE)
    grad = oracle.render_backward(cache, dLdA, FIELD)
    new, _, _ = oracle.adam_step(flat, grad, oracle.AdamState.zeros(flat.size), FIELD)
    lay = S.param_layout(FIELD)
    rng = np.random.default_rng(SEED + 1)
    top = np.argsort(-np.abs(grad))[:200]
    pick = np.concatenate([rng.choice(top, size=16, replace=False),
                           rng.choice(np.setdiff1d(np.nonzero(grad)[0], top), size=16, replace=False)])
    return {
        "what": "oracle training step: render (Eq. 1), MSE loss, backward, one Adam step (lr 1e-3)",
        "geometry": {"n_views": GEOM.n_views, "det_nu": GEOM.det_nu, "det_nv": GEOM.det_nv},
        "field": {"n_levels": FIELD.n_levels, "log2_T": FIELD.log2_T, "base_res": FIELD.base_res,
                  "max_res": FIELD.max_res, "hidden_layers": FIELD.hidden_layers},
        "view": VIEW, "n_samples": N, "seed": SEED, "pix": pix.tolist(),
        "A": A.tolist(), "loss": float(loss),
        "grad_norm": {k: float(np.linalg.norm(grad[v[0]:v[0] + v[1]])) for k, v in lay.items()
                      if not k.startswith("_")},
        "grad_max": float(np.abs(grad).max()),
        "grad_index": pick.tolist(), "grad_value": grad[pick].tolist(),
        "param_after_adam": new[pick].tolist(),
    }


if __name__ == "__main__":
    with open(os.path.join(HERE, "oracle_step.json"), "w") as fh:
        json.dump(expected(), fh, indent=1)
    print("wrote", os.path.join(HERE, "oracle_step.json"))
