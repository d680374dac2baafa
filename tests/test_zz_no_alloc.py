"""render_forward_noalloc: the forward pass for callers that cannot allocate device
memory when they call (plug-ins inside a host framework that owns every
allocation, real-time loops that forbid allocation after start-up). Both it and
render_forward launch the same kernels in the same order on the same inputs, so
their ray sums must agree bit for bit, call after call, although every call reuses
the same fixed scratch block; it must also refuse a batch that does not fit.

This file is named to be collected last, so that a run stopping at the first
failure has run every other test before it.
"""
import numpy as np
import pytest

import synthetic as S
from _cases import batch, field_cfg

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GEOM = S.GeometryConfig(n_views=6, det_nu=40, det_nv=36)


@pytest.mark.parametrize("precision", [S.PREC_F32, S.PREC_BF16])
def test_noalloc_forward_matches_workspace_forward_on_consecutive_calls(lib, precision):
    cfg = field_cfg(n_levels=16, hidden_layers=4, log2_T=12, max_res=256, precision=precision)
    field = lib.Field(cfg, params=S.init_params(cfg, 3, table_scale=0.5))
    geom = lib.Geometry.from_config(GEOM)
    for call, (view, R, N) in enumerate([(1, 300, 64), (4, 517, 45)]):
        pix = torch.as_tensor(batch(GEOM, view, R, seed=call, n_miss=3), device="cuda")
        ws = lib.workspace(lib.step_workspace_bytes(field, pix.numel(), N))
        a_ref = torch.empty(pix.numel(), device="cuda")
        lib.render_forward(field, geom, view, pix, N, a_ref, ws)
        a = torch.full((pix.numel(),), float("nan"), device="cuda")
        lib.render_forward_noalloc(field, geom, view, pix, N, a)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(a.cpu().numpy(), a_ref.cpu().numpy())


def test_noalloc_forward_rejects_a_batch_larger_than_its_scratch(lib):
    cfg = field_cfg()
    field = lib.Field(cfg, params=S.init_params(cfg, 0))
    geom = lib.Geometry.from_config(GEOM)
    pix = torch.zeros(60000, dtype=torch.int32, device="cuda")
    out = torch.empty(60000, device="cuda")
    with pytest.raises(lib.NHError) as e:
        lib.render_forward_noalloc(field, geom, 0, pix, 256, out)
    assert e.value.status == -3 and "fixed block" in str(e.value)
    with pytest.raises(lib.NHError) as e:
        lib.render_forward_noalloc(field, geom, 0, pix[:4], (1 << 20) + 1, out)
    assert e.value.status == -1
