"""Host-side checks of libnhcbct that need no GPU: the library builds and loads,
exports every function include/nhcbct.h declares, and its host logic (argument
validation, buffer layout, level resolutions, the per-view geometry table)
agrees with the oracle and the input generators. No call here launches a kernel."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import oracle
import synthetic as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def nh():
    from paper_2506_19742_gb300 import build, nhcbct
    build.build()
    return nhcbct


def _declared():
    src = open(os.path.join(ROOT, "include", "nhcbct.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:nh_status|void|int32_t|const char\*)\s+(\w+)\s*\(", src, flags=re.M)))


def test_library_exports_every_declared_symbol(nh):
    lib = nh.load()
    names = _declared()
    assert len(names) >= 30
    for n in names:
        assert hasattr(lib, n), n
        assert n in nh.EXPORTS, n
    assert lib.nh_version() == 101
    assert lib.nh_status_string(-3) == b"NH_ERR_SIZE_MISMATCH"


def _gdesc(nh, g: S.GeometryConfig, **kw):
    d = dict(n_views=g.n_views, angle0_rad=g.angle0_rad, span_rad=g.span_rad, dso_mm=g.dso_mm,
             dsd_mm=g.dsd_mm, det_nu=g.det_nu, det_nv=g.det_nv, det_du_mm=g.det_du_mm,
             det_dv_mm=g.det_dv_mm, vol_side_mm=g.vol_side_mm)
    d.update(kw)
    return nh.GeometryDesc(**d)


def test_view_table_is_bitwise_the_oracles(nh):
    for g in (S.GeometryConfig(n_views=50), S.GeometryConfig(n_views=100, det_nu=512, det_nv=512),
              S.GeometryConfig(n_views=7, angle0_rad=0.3, span_rad=1.1, det_nu=13, det_nv=9)):
        geom = nh.Geometry.from_config(g)
        tab, du, dv = geom.view_table()
        otab, odu, odv = oracle.view_table(g.n_views, g.angle0_rad, g.span_rad, g.dso_mm, g.dsd_mm,
                                           g.det_du_mm, g.det_dv_mm, g.vol_side_mm)
        assert np.array_equal(tab.view(np.uint32), otab.view(np.uint32))
        assert np.float32(du) == odu and np.float32(dv) == odv


def test_geometry_validation(nh):
    lib = nh.load()
    g = S.GeometryConfig()
    h = C.c_void_p()
    for bad in (dict(n_views=0), dict(det_nu=0), dict(dsd_mm=900.0), dict(vol_side_mm=-1.0),
                dict(dso_mm=100.0), dict(span_rad=float("nan"))):
        assert lib.geometry_create(C.byref(_gdesc(nh, g, **bad)), C.byref(h)) == -1, bad
    assert lib.geometry_create(None, C.byref(h)) == -1


def _fdesc(nh, f: S.FieldConfig):
    return nh.FieldDesc(f.n_levels, f.n_feat, f.log2_T, f.base_res, f.max_res, f.norm, f.ln_eps,
                        f.hidden_layers, f.width, f.precision, f.loss, f.lr, f.beta1, f.beta2,
                        f.adam_eps, f.loss_scale_init, f.growth_interval)


@pytest.mark.parametrize("wname", list(S.WORKLOADS))
def test_field_layout_matches_the_flat_parameter_format(nh, wname):
    f = S.WORKLOADS[wname].field
    lib = nh.load()
    sz = nh.FieldSizes()
    assert lib.field_query_sizes(C.byref(_fdesc(nh, f)), C.byref(sz)) == 0
    lay = S.param_layout(f)
    assert sz.n_params == lay["_total"][1]
    assert sz.n_table_params == lay["tables"][1]
    assert sz.off_gamma == lay["gamma"][0] and sz.off_beta == lay["beta"][0] and sz.off_mlp == lay["W0"][0]
    assert sz.bytes_params >= 4 * sz.n_params and sz.bytes_params % 16 == 0
    assert sz.bytes_tables_lp == (0 if f.precision == S.PREC_F32 else 2 * sz.n_table_params)


def _fake_field(nh, f):
    """A handle bound to fake (never dereferenced) device addresses."""
    lib = nh.load()
    fake = 1 << 40
    buf = nh.FieldBuffers(fake, fake, fake, fake, fake if f.precision else None, fake)
    h = C.c_void_p()
    assert lib.field_create(C.byref(_fdesc(nh, f)), C.byref(buf), C.byref(h)) == 0
    return h


def test_level_resolutions_and_validation(nh):
    lib = nh.load()
    for wname in ("tiny_fp32", "paper_fp32", "large_bf16"):
        f = S.WORKLOADS[wname].field
        h = _fake_field(nh, f)
        out = (C.c_int32 * 32)()
        assert lib.field_level_resolutions(h, out, 32) == 0
        assert list(out[: f.n_levels]) == oracle.level_resolutions(f.n_levels, f.base_res, f.max_res)
        lib.field_destroy(h)
    import dataclasses
    base = S.WORKLOADS["tiny_fp32"].field
    sz = nh.FieldSizes()
    for bad, code in ((dict(n_feat=4), -6), (dict(width=64), -6), (dict(n_levels=12), -6),
                      (dict(log2_T=30), -1), (dict(max_res=8), -1), (dict(norm=7), -1),
                      (dict(lr=0.0), -1), (dict(hidden_layers=0), -1), (dict(loss_scale_init=0.5), -1)):
        d = _fdesc(nh, dataclasses.replace(base, **bad))
        assert lib.field_query_sizes(C.byref(d), C.byref(sz)) == code, bad
    # misaligned and missing buffers
    d = _fdesc(nh, base)
    h = C.c_void_p()
    buf = nh.FieldBuffers(1 << 40, (1 << 40) + 4, 1 << 40, 1 << 40, None, 1 << 40)
    assert lib.field_create(C.byref(d), C.byref(buf), C.byref(h)) == -7
    buf = nh.FieldBuffers(1 << 40, None, 1 << 40, 1 << 40, None, 1 << 40)
    assert lib.field_create(C.byref(d), C.byref(buf), C.byref(h)) == -1


def test_batch_validation_rejects_before_any_launch(nh):
    lib = nh.load()
    f = S.WORKLOADS["tiny_fp32"].field
    h = _fake_field(nh, f)
    g = C.c_void_p()
    assert lib.geometry_create(C.byref(_gdesc(nh, S.GeometryConfig())), C.byref(g)) == 0
    need = C.c_size_t()
    assert lib.step_workspace_bytes(h, 1024, 64, C.byref(need)) == 0
    assert need.value >= 4 * (1024 * 2 + 1024 * 3)
    fake = 1 << 40
    ok = nh.RayBatch(0, 1024, fake, fake, 64)
    # workspace too small, misaligned, null; view, samples out of range; null pix
    assert lib.train_step(h, g, C.byref(ok), fake, fake, need.value - 1, None) == -3
    assert lib.train_step(h, g, C.byref(ok), fake, fake + 4, need.value, None) == -7
    assert lib.train_step(h, g, C.byref(ok), fake, None, need.value, None) == -1
    for bad in (nh.RayBatch(50, 1024, fake, fake, 64), nh.RayBatch(-1, 1024, fake, fake, 64),
                nh.RayBatch(0, 1024, fake, fake, 0), nh.RayBatch(0, -5, fake, fake, 64),
                nh.RayBatch(0, 1024, None, fake, 64), nh.RayBatch(0, 1024, fake, None, 64)):
        assert lib.train_step(h, g, C.byref(bad), fake, fake, need.value, None) == -1
    assert lib.train_step(None, g, C.byref(ok), fake, fake, need.value, None) == -1
    buf = C.create_string_buffer(256)
    lib.nh_last_error(buf, 256)
    assert b"train_step" in buf.value
    assert lib.query_volume(h, 0, fake, None) == -1
    assert lib.project(g, fake, 16, 0, fake, None) == -1
    n = C.c_size_t()
    assert lib.field_export_bytes(h, 2 | 4, C.byref(n)) == 0
    assert n.value == 4 * (S.param_layout(f)["_total"][1] - S.param_layout(f)["gamma"][0])
    assert lib.field_export_bytes(h, 16, C.byref(n)) == -1
    lib.field_destroy(h)
    lib.geometry_destroy(g)


def test_ssim_workspace_and_validation_reject_before_any_launch(nh):
    """ssim3d's host checks: window sizes 11..1024, positive finite data range,
    8-byte alignment, workspace size; every bad call returns before touching the
    (fake) device pointers."""
    lib = nh.load()
    n = C.c_size_t()
    for D, M in ((11, 1), (128, 118)):
        assert lib.ssim3d_workspace_bytes(D, C.byref(n)) == 0
        assert n.value == 8 * (5 * D * D * M + 5 * D * M * M + 1024)
    for bad in (10, 0, -3, 1025):
        assert lib.ssim3d_workspace_bytes(bad, C.byref(n)) == -1
    assert lib.ssim3d_workspace_bytes(11, None) == -1
    assert lib.ssim3d_workspace_bytes(64, C.byref(n)) == 0
    need = n.value
    fake = 1 << 40
    assert lib.ssim3d(fake, fake, 64, 1.0, fake, None, fake, need - 1, None) == -3
    assert lib.ssim3d(fake, fake, 64, 1.0, fake, fake + 4, fake, need, None) == -7
    assert lib.ssim3d(fake, fake, 64, 1.0, fake + 4, None, fake, need, None) == -7
    assert lib.ssim3d(fake, fake, 64, 1.0, fake, None, fake + 12, need, None) == -7
    for dr in (0.0, -1.0, float("nan"), float("inf")):
        assert lib.ssim3d(fake, fake, 64, dr, fake, None, fake, need, None) == -1
    assert lib.ssim3d(fake, fake, 10, 1.0, fake, None, fake, need, None) == -1
    assert lib.ssim3d(None, fake, 64, 1.0, fake, None, fake, need, None) == -1
    assert lib.ssim3d(fake, fake, 64, 1.0, None, None, fake, need, None) == -1
    buf = C.create_string_buffer(256)
    lib.nh_last_error(buf, 256)
    assert b"ssim3d" in buf.value


def test_checkpoint_config_hash_tracks_the_field_description(nh):
    """Checkpoints load only into a field of the same description: the hash is a
    pure function of the description's values and changes with any of them."""
    import dataclasses
    f = S.WORKLOADS["tiny_fp32"].field
    h0 = nh.config_hash(_fdesc(nh, f))
    assert h0 == nh.config_hash(_fdesc(nh, dataclasses.replace(f)))
    assert len(h0) == 16 and int(h0, 16) >= 0
    seen = {h0}
    for change in (dict(log2_T=15), dict(n_levels=4), dict(norm=S.NORM_NONE), dict(precision=S.PREC_BF16),
                   dict(lr=2e-3), dict(loss=S.LOSS_L1), dict(hidden_layers=4)):
        h = nh.config_hash(_fdesc(nh, dataclasses.replace(f, **change)))
        assert h not in seen, change
        seen.add(h)


def test_every_declared_function_is_documented():
    """Each entry point of include/nhcbct.h carries its own comment block (meaning
    of the arguments, layout, ownership, errors) directly above it, or shares the
    block of the declaration group it belongs to."""
    lines = open(os.path.join(ROOT, "include", "nhcbct.h")).read().splitlines()
    decl = re.compile(r"^\s*(?:nh_status|void|int32_t|const char\*)\s+(\w+)\s*\(")
    undocumented = []
    for i, line in enumerate(lines):
        m = decl.match(line)
        if not m:
            continue
        j = i - 1
        while j >= 0 and (decl.match(lines[j]) or not lines[j].strip() or lines[j].rstrip().endswith(",")
                          or lines[j].strip().endswith(");")):
            j -= 1
        if j < 0 or not lines[j].rstrip().endswith("*/"):
            undocumented.append(m.group(1))
    assert not undocumented, undocumented


def test_point_stage_and_export_validation_rejects_before_any_launch(nh):
    """Host checks of the point, stage-probe, export / import and render entry
    points: null, negative, misaligned and undersized arguments return their status
    codes without touching the (fake) device addresses."""
    lib = nh.load()
    f = S.WORKLOADS["tiny_fp32"].field
    h = _fake_field(nh, f)
    g = C.c_void_p()
    assert lib.geometry_create(C.byref(_gdesc(nh, S.GeometryConfig())), C.byref(g)) == 0
    fake = 1 << 40
    need = C.c_size_t()
    # voxel-loss pre-training (Eq. 2) and its workspace
    assert lib.points_workspace_bytes(h, 4096, C.byref(need)) == 0 and need.value % 256 == 0
    assert lib.points_workspace_bytes(h, -1, C.byref(need)) == -1
    assert lib.points_workspace_bytes(None, 16, C.byref(need)) == -1
    assert lib.points_workspace_bytes(h, 4096, C.byref(need)) == 0
    for fn in (lib.fit_points_step, lib.fit_points_backward):
        assert fn(None, 16, fake, fake, fake, fake, need.value, None) == -1
        assert fn(h, -1, fake, fake, fake, fake, need.value, None) == -1
        assert fn(h, 4096, None, fake, fake, fake, need.value, None) == -1
        assert fn(h, 4096, fake + 2, fake, fake, fake, need.value, None) == -7
        assert fn(h, 4096, fake, fake, fake, None, need.value, None) == -1
        assert fn(h, 4096, fake, fake, fake, fake + 64, need.value, None) == -7
        assert fn(h, 4096, fake, fake, fake, fake, need.value - 1, None) == -3
    # queries
    assert lib.query_points(None, 8, fake, fake, None) == -1
    assert lib.query_points(h, -1, fake, fake, None) == -1
    assert lib.query_points(h, 8, None, fake, None) == -1
    assert lib.query_points(h, 0, None, None, None) == 0          # nothing to do, nothing launched
    assert lib.query_volume(h, -4, fake, None) == -1
    # stage probes
    assert lib.sample_rays(None, 0, 4, fake, 16, 0, fake, fake, None) == -1
    assert lib.sample_rays(g, 0, 4, None, 16, 0, fake, fake, None) == -1
    assert lib.sample_rays(g, 50, 4, fake, 16, 0, fake, fake, None) == -1
    assert lib.sample_rays(g, 0, 4, fake, 0, 0, fake, fake, None) == -1
    assert lib.hash_corners(h, 4, None, fake, fake, None) == -1
    assert lib.hash_corners(h, -4, fake, fake, fake, None) == -1
    assert lib.encode_points(h, 4, fake, None, None) == -1
    assert lib.encode_points(h, -4, fake, fake, None) == -1
    assert lib.scatter_points(h, 4, fake, None, None) == -1
    assert lib.scatter_points(h, -4, fake, fake, None) == -1
    assert lib.scatter_points(h, 4, fake, fake + 8, None) == -7
    # export / import of parts
    n = C.c_size_t()
    assert lib.field_export_bytes(h, 2 | 4, C.byref(n)) == 0
    assert lib.field_export(h, 2 | 4, None, n.value, None) == -1
    assert lib.field_export(h, 2 | 4, fake, n.value - 4, None) == -3
    assert lib.field_import(h, 2 | 4, fake, n.value - 4, None) == -3
    assert lib.field_export(None, 2 | 4, fake, n.value, None) == -1
    assert lib.field_import(h, 16, fake, n.value, None) == -1
    assert lib.field_set_channel_mask(h, None, f.n_levels * f.n_feat, None) == -1
    mask = (C.c_float * 64)()
    assert lib.field_set_channel_mask(h, mask, f.n_levels * f.n_feat - 1, None) == -3
    # render_forward / render_backward share the batch checks; backward needs dL/dA
    assert lib.step_workspace_bytes(h, 64, 32, C.byref(need)) == 0
    ok = nh.RayBatch(0, 64, fake, fake, 32)
    assert lib.render_forward(h, g, C.byref(ok), None, fake, need.value, None) == -1
    assert lib.render_backward(h, g, C.byref(ok), None, fake, need.value, None) == -1
    assert lib.render_forward(h, g, C.byref(ok), fake, fake, need.value - 1, None) == -3
    assert lib.render_backward(h, g, C.byref(nh.RayBatch(0, 64, fake, fake, 0)), fake, fake, need.value, None) == -1
    lib.field_destroy(h)
    lib.geometry_destroy(g)


def test_channel_mask_selection_validation_rejects_before_any_launch(nh):
    """Host checks of the FFT channel-mask selection (Sec. 2.3): grid size, cutoff,
    threshold, null, misaligned and undersized buffers return their status codes
    without touching the (fake) device addresses; the workspace is two complex FP64 planes of G^3 x L F values plus the
    channel means."""
    lib = nh.load()
    f = S.WORKLOADS["paper_fp32"].field
    h = _fake_field(nh, f)
    fake = 1 << 40
    need = C.c_size_t()
    assert lib.channel_mask_workspace_bytes(h, 64, C.byref(need)) == 0
    D = f.n_levels * f.n_feat
    assert need.value >= 2 * 16 * 64 ** 3 * D + 8 * D and need.value % 256 == 0
    assert lib.channel_mask_workspace_bytes(h, 1, C.byref(need)) == -1
    assert lib.channel_mask_workspace_bytes(h, 129, C.byref(need)) == -1
    assert lib.channel_mask_workspace_bytes(None, 64, C.byref(need)) == -1
    assert lib.channel_mask_workspace_bytes(h, 64, C.byref(need)) == 0
    sel = lib.field_select_channel_mask
    assert sel(None, 64, 0.25, 0.85, 1, fake, fake, fake, need.value, None) == -1
    assert sel(h, 64, 0.25, 0.85, 1, None, fake, fake, need.value, None) == -1
    assert sel(h, 64, 0.25, 0.85, 1, fake, fake, None, need.value, None) == -1
    assert sel(h, 1, 0.25, 0.85, 1, fake, fake, fake, need.value, None) == -1
    assert sel(h, 200, 0.25, 0.85, 1, fake, fake, fake, need.value, None) == -1
    assert sel(h, 64, -0.1, 0.85, 1, fake, fake, fake, need.value, None) == -1
    assert sel(h, 64, float("nan"), 0.85, 1, fake, fake, fake, need.value, None) == -1
    assert sel(h, 64, 0.25, float("inf"), 1, fake, fake, fake, need.value, None) == -1
    assert sel(h, 64, 0.25, 0.85, 1, fake + 4, fake, fake, need.value, None) == -7
    assert sel(h, 64, 0.25, 0.85, 1, fake, fake + 2, fake, need.value, None) == -7
    assert sel(h, 64, 0.25, 0.85, 1, fake, fake, fake + 128, need.value, None) == -7
    assert sel(h, 64, 0.25, 0.85, 1, fake, fake, fake, need.value - 1, None) == -3
    lib.field_destroy(h)


def test_roofline_probe_validation_rejects_before_any_launch(nh):
    """Host checks of the roofline probes (random gather, float2 and packed 16-bit
    reductions, streaming read): null, non-power-of-two, oversized, misaligned and
    wrong-format arguments return their status codes without touching the (fake)
    device addresses."""
    lib = nh.load()
    fake = 1 << 40
    done = C.c_int64()
    assert lib.probe_random_red16(None, 1 << 20, 1, 1024, C.byref(done), None) == -1
    assert lib.probe_random_red16(fake, 1 << 20, 1, 1024, None, None) == -1
    assert lib.probe_random_red16(fake, 3 << 20, 1, 1024, C.byref(done), None) == -1
    assert lib.probe_random_red16(fake, 1 << 33, 2, 1024, C.byref(done), None) == -1
    assert lib.probe_random_red16(fake, 1 << 20, 0, 1024, C.byref(done), None) == -1   # FP32 is not packed
    assert lib.probe_random_red16(fake, 1 << 20, 1, -1, C.byref(done), None) == -1
    assert lib.probe_random_red16(fake + 2, 1 << 20, 2, 1024, C.byref(done), None) == -7
    assert lib.probe_random_red(fake, 1 << 20, 1024, None, None) == -1
    assert lib.probe_random_red(fake, 1000, 1024, C.byref(done), None) == -1
    assert lib.probe_random_red(fake + 4, 1 << 20, 1024, C.byref(done), None) == -7
    assert lib.probe_random_gather(fake, 1 << 20, 6, 1024, fake, C.byref(done), None) == -1
    assert lib.probe_random_gather(fake + 4, 1 << 20, 8, 1024, fake, C.byref(done), None) == -7
    assert lib.probe_l2_read(fake, 1000, 1, fake, None) == -1
    assert lib.probe_l2_read(fake + 8, 1024, 1, fake, None) == -7
    assert lib.probe_l2_read(fake, 1024, 0, fake, None) == -1
