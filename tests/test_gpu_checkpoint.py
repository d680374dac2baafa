"""Checkpoint / resume (Field.save / Field.load over the caller-owned buffers) and
run-to-run repeatability of the training step.

A checkpoint holds the parameters, both Adam moments and the device state block
(Adam step count, loss scale, growth counter, channel mask). A field restored from
it takes the next step with the same bits as the field that wrote it: the forward,
the ray sums and the loss are summed in a fixed order. Only the gradient sums
(atomics into the tables and the CTA accumulators) may differ in order from run to
run."""
import numpy as np
import pytest

import synthetic as S

pytestmark = pytest.mark.gpu


def _batches(lib, torch, w, n, seed):
    geom = lib.Geometry.from_config(w.geometry)
    g = w.geometry
    hp = torch.empty(g.n_views * g.det_nv * g.det_nu, device="cuda")
    lib.project(geom, torch.ones(32 ** 3, device="cuda"), 1, hp)
    hit = hp.view(g.n_views, -1).cpu().numpy() > 0
    cands = [np.nonzero(hit[v])[0] for v in range(g.n_views)]
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        view, pix = S.pick_rays(rng, g.n_views, cands, w.n_rays)
        out.append((view, torch.from_numpy(pix).cuda(), torch.rand(w.n_rays, device="cuda", generator=None)))
    return geom, out


@pytest.mark.parametrize("wname", ["tiny_fp32", "tiny_bf16", "tiny_f16"])
def test_checkpoint_resumes_training_with_the_same_bits(lib, wname, tmp_path):
    import torch
    torch.manual_seed(0)
    w = S.WORKLOADS[wname]
    geom, batches = _batches(lib, torch, w, 8, 1)
    a = lib.Field(w.field, params=S.init_params(w.field, 0))
    mask = np.ones(w.field.n_levels * w.field.n_feat, dtype=np.float32)
    mask[-3:] = 0.0
    a.set_channel_mask(mask)
    ws = lib.workspace(lib.step_workspace_bytes(a, w.n_rays, w.n_samples))
    loss = torch.zeros(1, device="cuda")
    for view, pix, am in batches[:4]:
        lib.train_step(a, geom, view, pix, am, w.n_samples, loss, ws)
    path = str(tmp_path / "field.npz")
    a.save(path)
    snap = {k: getattr(a, k)[: a.n_params].clone() for k in ("params", "adam_m", "adam_v")}
    state = a.state.clone()

    b = lib.Field(w.field, params=S.init_params(w.field, 1))     # other initial values
    b.load(path)
    for k, v in snap.items():
        assert torch.equal(getattr(b, k)[: b.n_params], v), k
    assert torch.equal(b.state, state)
    assert float(b.grads.abs().max()) == 0.0
    assert b.poll_status() == a.poll_status()
    if a.tables_lp is not None:
        assert torch.equal(b.tables_lp, a.tables_lp)

    la, lb = [], []
    for view, pix, am in batches[4:]:
        lib.train_step(a, geom, view, pix, am, w.n_samples, loss, ws)
        la.append(float(loss.item()))
        lib.train_step(b, geom, view, pix, am, w.n_samples, loss, ws)
        lb.append(float(loss.item()))
    assert la[0] == lb[0]                                     # same state, fixed-order sums
    np.testing.assert_allclose(lb, la, rtol=1e-4)             # later steps: gradient sum order only
    assert a.poll_status()[1:] == b.poll_status()[1:]         # loss scale and step count


def test_checkpoint_refuses_another_field_description(lib, tmp_path):
    import dataclasses
    w = S.WORKLOADS["tiny_fp32"]
    a = lib.Field(w.field, params=S.init_params(w.field, 0))
    path = str(tmp_path / "field.npz")
    a.save(path)
    for change in (dict(log2_T=w.field.log2_T + 1), dict(lr=2e-3), dict(precision=S.PREC_BF16)):
        other = lib.Field(dataclasses.replace(w.field, **change))
        with pytest.raises(ValueError):
            other.load(path)
    np.savez(str(tmp_path / "junk.npz"), format=np.array("something-else"))
    with pytest.raises(ValueError):
        a.load(str(tmp_path / "junk.npz"))


@pytest.mark.parametrize("wname", ["paper_fp32", "paper_bf16"])
def test_training_step_repeats_up_to_gradient_sum_order(lib, wname, tmp_path):
    """The same step from the same state twice: the loss is bit-identical, and the
    gradients differ only by the order of their atomic sums, within 1e-3 of the
    largest entry of each part (hash tables, LN, MLP)."""
    import torch
    w = S.WORKLOADS[wname]
    geom, batches = _batches(lib, torch, w, 2, 3)
    f = lib.Field(w.field, params=S.init_params(w.field, 0))
    ws = lib.workspace(lib.step_workspace_bytes(f, w.n_rays, w.n_samples))
    loss = torch.zeros(1, device="cuda")
    lib.train_step(f, geom, *batches[0], w.n_samples, loss, ws)
    view, pix, am = batches[1]
    runs = []
    for _ in range(2):
        f.grads.zero_()
        lib.accumulate_step(f, geom, view, pix, am, w.n_samples, loss, ws)
        runs.append((float(loss.item()), f.flat_grads().clone()))
    assert runs[0][0] == runs[1][0]
    g1, g2 = runs[0][1], runs[1][1]
    lay = S.param_layout(w.field)
    n_tab = lay["gamma"][0]
    for lo, hi in ((0, n_tab), (n_tab, lay["_total"][1])):
        scale = float(g1[lo:hi].abs().max())
        assert scale > 0.0
        assert float((g1[lo:hi] - g2[lo:hi]).abs().max()) <= 1e-3 * scale
