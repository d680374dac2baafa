"""Python binding of libnhcbct (ctypes): argument marshalling only.

Every computation runs in the CUDA library; PyTorch supplies device memory and
streams. The functions named like the C ABI (``train_step``, ``render_forward``,
``query_volume``, ``project`` ...) take torch tensors and forward their device
pointers and the current CUDA stream. ``Geometry`` and ``Field`` own the
caller-side buffers the library asks for. Loading fails loudly if the built
library is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnhcbct.so")

NORM_NONE, NORM_LN, NORM_LN_PER_LEVEL = 0, 1, 2
PREC_F32, PREC_BF16, PREC_F16 = 0, 1, 2
LOSS_MSE, LOSS_L1 = 0, 1
PART_HASH, PART_LN, PART_MLP, PART_ADAM = 1, 2, 4, 8
FLAG_NONFINITE, FLAG_SKIPPED = 1, 2
STATUS = {0: "NH_OK", -1: "NH_ERR_INVALID_ARG", -2: "NH_ERR_CUDA", -3: "NH_ERR_SIZE_MISMATCH",
          -4: "NH_ERR_NONFINITE", -5: "NH_ERR_TIMEOUT", -6: "NH_ERR_UNSUPPORTED", -7: "NH_ERR_ALIGNMENT"}


class NHError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        super().__init__(f"{where}: {STATUS.get(status, status)}: {detail}")
        self.status = status


class GeometryDesc(C.Structure):
    _fields_ = [("n_views", C.c_int32), ("angle0_rad", C.c_double), ("span_rad", C.c_double),
                ("dso_mm", C.c_double), ("dsd_mm", C.c_double), ("det_nu", C.c_int32),
                ("det_nv", C.c_int32), ("det_du_mm", C.c_double), ("det_dv_mm", C.c_double),
                ("vol_side_mm", C.c_double)]


class FieldDesc(C.Structure):
    _fields_ = [("n_levels", C.c_int32), ("n_feat", C.c_int32), ("log2_T", C.c_int32),
                ("base_res", C.c_int32), ("max_res", C.c_int32), ("norm", C.c_int32),
                ("ln_eps", C.c_float), ("hidden_layers", C.c_int32), ("width", C.c_int32),
                ("precision", C.c_int32), ("loss", C.c_int32), ("lr", C.c_float),
                ("beta1", C.c_float), ("beta2", C.c_float), ("adam_eps", C.c_float),
                ("loss_scale_init", C.c_float), ("growth_interval", C.c_int32)]


class FieldSizes(C.Structure):
    _fields_ = [(n, C.c_uint64) for n in (
        "n_params", "n_table_params", "off_gamma", "off_beta", "off_mlp", "bytes_params",
        "bytes_grads", "bytes_adam_m", "bytes_adam_v", "bytes_tables_lp", "bytes_state")]


class FieldBuffers(C.Structure):
    _fields_ = [("params", C.c_void_p), ("grads", C.c_void_p), ("adam_m", C.c_void_p),
                ("adam_v", C.c_void_p), ("tables_lp", C.c_void_p), ("state", C.c_void_p)]


class RayBatch(C.Structure):
    _fields_ = [("view", C.c_int32), ("n_rays", C.c_int32), ("pix", C.c_void_p),
                ("a_meas", C.c_void_p), ("n_samples", C.c_int32), ("jitter_seed", C.c_uint64)]


_P = C.c_void_p
_I = C.c_int32
_SZ = C.c_size_t
_SIGS = {
    "nh_status_string": (C.c_char_p, [_I]),
    "nh_last_error": (_I, [C.c_char_p, _SZ]),
    "nh_version": (_I, []),
    "geometry_create": (_I, [C.POINTER(GeometryDesc), C.POINTER(_P)]),
    "geometry_destroy": (None, [_P]),
    "geometry_view_table": (_I, [_P, C.POINTER(C.c_float), _SZ]),
    "field_query_sizes": (_I, [C.POINTER(FieldDesc), C.POINTER(FieldSizes)]),
    "field_create": (_I, [C.POINTER(FieldDesc), C.POINTER(FieldBuffers), C.POINTER(_P)]),
    "field_destroy": (None, [_P]),
    "field_reset_state": (_I, [_P, _P]),
    "field_refresh_lowp": (_I, [_P, _P]),
    "field_set_channel_mask": (_I, [_P, C.POINTER(C.c_float), _I, _P]),
    "field_level_resolutions": (_I, [_P, C.POINTER(_I), _I]),
    "channel_mask_workspace_bytes": (_I, [_P, _I, C.POINTER(_SZ)]),
    "field_select_channel_mask": (_I, [_P, _I, C.c_double, C.c_double, _I, _P, _P, _P, _SZ, _P]),
    "field_export_bytes": (_I, [_P, C.c_uint32, C.POINTER(_SZ)]),
    "field_export": (_I, [_P, C.c_uint32, _P, _SZ, _P]),
    "field_import": (_I, [_P, C.c_uint32, _P, _SZ, _P]),
    "field_poll_status": (_I, [_P, _P, C.POINTER(C.c_uint32), C.POINTER(C.c_float), C.POINTER(_I)]),
    "step_workspace_bytes": (_I, [_P, _I, _I, C.POINTER(_SZ)]),
    "points_workspace_bytes": (_I, [_P, _I, C.POINTER(_SZ)]),
    "train_step": (_I, [_P, _P, C.POINTER(RayBatch), _P, _P, _SZ, _P]),
    "accumulate_step": (_I, [_P, _P, C.POINTER(RayBatch), _P, _P, _SZ, _P]),
    "train_step_host": (_I, [_P, _P, _I, _I, _P, _P, _I, _P, _P, _SZ, _P]),
    "render_forward": (_I, [_P, _P, C.POINTER(RayBatch), _P, _P, _SZ, _P]),
    "render_backward": (_I, [_P, _P, C.POINTER(RayBatch), _P, _P, _SZ, _P]),
    "render_forward_noalloc": (_I, [_P, _P, C.POINTER(RayBatch), _P, _P]),
    "optimizer_step": (_I, [_P, _P]),
    "fit_points_step": (_I, [_P, _I, _P, _P, _P, _P, _SZ, _P]),
    "fit_points_backward": (_I, [_P, _I, _P, _P, _P, _P, _SZ, _P]),
    "query_points": (_I, [_P, _I, _P, _P, _P]),
    "query_volume": (_I, [_P, _I, _P, _P]),
    "project": (_I, [_P, _P, _I, _I, _P, _P]),
    "volume_mse": (_I, [_P, _P, C.c_int64, _P, _P, _SZ, _P]),
    "ssim3d": (_I, [_P, _P, _I, C.c_double, _P, _P, _P, _SZ, _P]),
    "ssim3d_workspace_bytes": (_I, [_I, C.POINTER(_SZ)]),
    "launch_info": (_I, [C.POINTER(_I), _I]),
    "sample_rays": (_I, [_P, _I, _I, _P, _I, C.c_uint64, _P, _P, _P]),
    "hash_corners": (_I, [_P, _I, _P, _P, _P, _P]),
    "encode_points": (_I, [_P, _I, _P, _P, _P]),
    "scatter_points": (_I, [_P, _I, _P, _P, _P]),
    "probe_l2_read": (_I, [_P, C.c_uint64, _I, _P, _P]),
    "probe_random_gather": (_I, [_P, C.c_uint64, _I, C.c_int64, _P, C.POINTER(C.c_int64), _P]),
    "probe_random_red": (_I, [_P, C.c_uint64, C.c_int64, C.POINTER(C.c_int64), _P]),
    "probe_random_red16": (_I, [_P, C.c_uint64, _I, C.c_int64, C.POINTER(C.c_int64), _P]),
}
EXPORTS = tuple(_SIGS)

_lib = None


def load(path: str = LIB_PATH):
    """Loads libnhcbct.so (built by ``paper_2506_19742_gb300.build``); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libnhcbct.so not found at {path}: build it with "
                           "`python -m paper_2506_19742_gb300.build` (no CPU fallback exists)")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status: int, where: str):
    if status != 0:
        buf = C.create_string_buffer(512)
        load().nh_last_error(buf, 512)
        raise NHError(status, where, buf.value.decode(errors="replace"))


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream=None):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _dev(t, dtype, name):
    if t is None:
        return None
    if not (t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise ValueError(f"{name}: expected a contiguous CUDA {dtype} tensor")
    return t


# ---------------------------------------------------------------------------- handles
class Geometry:
    """Cone-beam scan geometry (host metadata only)."""

    def __init__(self, n_views=50, angle0_rad=0.0, span_rad=2 * 3.141592653589793, dso_mm=1000.0,
                 dsd_mm=1500.0, det_nu=64, det_nv=64, det_du_mm=None, det_dv_mm=None,
                 vol_side_mm=256.0, det_side_mm=700.0):
        lib = load()
        du = det_side_mm / det_nu if det_du_mm is None else det_du_mm
        dv = det_side_mm / det_nv if det_dv_mm is None else det_dv_mm
        self.desc = GeometryDesc(n_views, angle0_rad, span_rad, dso_mm, dsd_mm, det_nu, det_nv, du, dv,
                                 vol_side_mm)
        h = C.c_void_p()
        _check(lib.geometry_create(C.byref(self.desc), C.byref(h)), "geometry_create")
        self.handle = h
        self.n_views, self.nu, self.nv = n_views, det_nu, det_nv

    @classmethod
    def from_config(cls, g):
        return cls(g.n_views, g.angle0_rad, g.span_rad, g.dso_mm, g.dsd_mm, g.det_nu, g.det_nv,
                   g.det_du_mm, g.det_dv_mm, g.vol_side_mm)

    def view_table(self):
        n = 12 * self.n_views + 2
        buf = (C.c_float * n)()
        _check(load().geometry_view_table(self.handle, buf, n), "geometry_view_table")
        import numpy as np
        a = np.frombuffer(buf, dtype=np.float32).copy()
        return a[:-2].reshape(self.n_views, 12), a[-2], a[-1]

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.geometry_destroy(self.handle)
            self.handle = None


CHECKPOINT_FORMAT = "nhcbct-field-1"


def _desc_json(desc) -> str:
    import json
    return json.dumps({name: getattr(desc, name) for name, _ in desc._fields_}, sort_keys=True)


def config_hash(desc) -> str:
    """sha256 (16 hex digits) of a field description's values: checkpoints load
    only into a field of the same description."""
    import hashlib
    return hashlib.sha256(_desc_json(desc).encode()).hexdigest()[:16]


def _stream_sync(stream=None):
    (stream if stream is not None else torch.cuda.current_stream()).synchronize()


class Field:
    """Hash grid + Normalized Hash Encoder + MLP with its caller-owned device buffers."""

    def __init__(self, cfg, device="cuda", params=None):
        lib = load()
        self.cfg = cfg
        self.desc = FieldDesc(cfg.n_levels, cfg.n_feat, cfg.log2_T, cfg.base_res, cfg.max_res, cfg.norm,
                              cfg.ln_eps, cfg.hidden_layers, cfg.width, cfg.precision, cfg.loss, cfg.lr,
                              cfg.beta1, cfg.beta2, cfg.adam_eps, cfg.loss_scale_init, cfg.growth_interval)
        self.sizes = FieldSizes()
        _check(lib.field_query_sizes(C.byref(self.desc), C.byref(self.sizes)), "field_query_sizes")
        nf = self.sizes.bytes_params // 4
        self.params = torch.zeros(nf, dtype=torch.float32, device=device)
        self.grads = torch.zeros(nf, dtype=torch.float32, device=device)
        self.adam_m = torch.zeros(nf, dtype=torch.float32, device=device)
        self.adam_v = torch.zeros(nf, dtype=torch.float32, device=device)
        lp = self.sizes.bytes_tables_lp
        lp_dtype = torch.bfloat16 if cfg.precision == PREC_BF16 else torch.float16
        self.tables_lp = torch.zeros(lp // 2, dtype=lp_dtype, device=device) if lp else None
        self.state = torch.zeros(self.sizes.bytes_state // 4, dtype=torch.float32, device=device)
        self.buffers = FieldBuffers(self.params.data_ptr(), self.grads.data_ptr(), self.adam_m.data_ptr(),
                                    self.adam_v.data_ptr(),
                                    self.tables_lp.data_ptr() if self.tables_lp is not None else None,
                                    self.state.data_ptr())
        h = C.c_void_p()
        _check(lib.field_create(C.byref(self.desc), C.byref(self.buffers), C.byref(h)), "field_create")
        self.handle = h
        self.n_params = int(self.sizes.n_params)
        if params is not None:
            self.load_params(params)
        else:
            self.reset_state()

    def load_params(self, flat):
        """Copies a flat float32 parameter vector in and resets the optimizer state."""
        t = torch.as_tensor(flat, dtype=torch.float32)
        self.params[: self.n_params].copy_(t.to(self.params.device))
        self.reset_state()

    def reset_state(self, stream=None):
        _check(load().field_reset_state(self.handle, _stream(stream)), "field_reset_state")

    def refresh_lowp(self, stream=None):
        _check(load().field_refresh_lowp(self.handle, _stream(stream)), "field_refresh_lowp")

    def set_channel_mask(self, mask, stream=None):
        import numpy as np
        m = np.ascontiguousarray(mask, dtype=np.float32)
        _check(load().field_set_channel_mask(self.handle, m.ctypes.data_as(C.POINTER(C.c_float)), len(m),
                                             _stream(stream)), "field_set_channel_mask")

    def level_resolutions(self):
        out = (C.c_int32 * 32)()
        _check(load().field_level_resolutions(self.handle, out, 32), "field_level_resolutions")
        return list(out[: self.cfg.n_levels])

    def poll_status(self, stream=None):
        flags, scale, step = C.c_uint32(), C.c_float(), C.c_int32()
        _check(load().field_poll_status(self.handle, _stream(stream), C.byref(flags), C.byref(scale),
                                        C.byref(step)), "field_poll_status")
        return flags.value, scale.value, step.value

    def export_bytes(self, parts):
        n = C.c_size_t()
        _check(load().field_export_bytes(self.handle, parts, C.byref(n)), "field_export_bytes")
        return n.value

    def export(self, parts, stream=None):
        out = torch.empty(self.export_bytes(parts) // 4, dtype=torch.float32, device=self.params.device)
        _check(load().field_export(self.handle, parts, _ptr(out), out.numel() * 4, _stream(stream)),
               "field_export")
        return out

    def import_(self, parts, blob, stream=None):
        blob = _dev(blob, torch.float32, "blob")
        _check(load().field_import(self.handle, parts, _ptr(blob), blob.numel() * 4, _stream(stream)),
               "field_import")

    def flat_params(self):
        return self.params[: self.n_params]

    def flat_grads(self):
        return self.grads[: self.n_params]

    # ------------------------------------------------------------ checkpoint / resume
    def save(self, path, stream=None):
        """Writes a checkpoint (.npz): the field description and its hash, the
        parameters, both Adam moments and the device state block (Adam step count,
        loss scale and its growth counter, channel mask). Gradients are not kept:
        a checkpoint is taken between steps. load() of it resumes training with the
        same bits."""
        import numpy as np
        _stream_sync(stream)
        np.savez(path, format=np.array(CHECKPOINT_FORMAT), config=np.array(_desc_json(self.desc)),
                 config_hash=np.array(config_hash(self.desc)),
                 params=self.params[: self.n_params].cpu().numpy(),
                 adam_m=self.adam_m[: self.n_params].cpu().numpy(),
                 adam_v=self.adam_v[: self.n_params].cpu().numpy(),
                 state=self.state.cpu().numpy())

    def load(self, path, stream=None):
        """Restores a checkpoint written by save() into this field, which must have
        been created with the same description (checked by its hash). Zeroes the
        gradients and refreshes the 16-bit table copy."""
        import numpy as np
        with np.load(path) as z:
            if str(z["format"]) != CHECKPOINT_FORMAT:
                raise ValueError(f"{path}: not a {CHECKPOINT_FORMAT} checkpoint")
            if str(z["config_hash"]) != config_hash(self.desc):
                raise ValueError(f"{path}: checkpoint of another field description: {z['config']}")
            n = self.n_params
            for name, buf in (("params", self.params), ("adam_m", self.adam_m), ("adam_v", self.adam_v)):
                a = z[name]
                if a.shape != (n,) or a.dtype != np.float32:
                    raise ValueError(f"{path}: {name} holds {a.shape} {a.dtype}, need ({n},) float32")
                buf[:n].copy_(torch.from_numpy(a).to(buf.device))
            st = z["state"]
            if st.shape != tuple(self.state.shape) or st.dtype != np.float32:
                raise ValueError(f"{path}: state block of another layout")
            self.state.copy_(torch.from_numpy(st).to(self.state.device))
        self.grads.zero_()
        if self.tables_lp is not None:
            self.refresh_lowp(stream)
        _stream_sync(stream)

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.field_destroy(self.handle)
            self.handle = None


# ---------------------------------------------------------------------------- workspaces
def step_workspace_bytes(field: Field, n_rays: int, n_samples: int) -> int:
    n = C.c_size_t()
    _check(load().step_workspace_bytes(field.handle, n_rays, n_samples, C.byref(n)), "step_workspace_bytes")
    return n.value


def points_workspace_bytes(field: Field, n_pts: int) -> int:
    n = C.c_size_t()
    _check(load().points_workspace_bytes(field.handle, n_pts, C.byref(n)), "points_workspace_bytes")
    return n.value


def workspace(nbytes: int, device="cuda"):
    """A 256-byte aligned device workspace (torch allocations are 512-byte aligned)."""
    return torch.empty(max(1, (nbytes + 3) // 4), dtype=torch.float32, device=device)


def _batch(view, pix, a_meas, n_samples, jitter_seed=0):
    """jitter_seed 0: midpoint samples; otherwise stratified jitter drawn from it."""
    pix = _dev(pix, torch.int32, "pix")
    a_meas = _dev(a_meas, torch.float32, "a_meas")
    n = 0 if pix is None else pix.numel()
    return RayBatch(int(view), n, pix.data_ptr() if pix is not None else None,
                    a_meas.data_ptr() if a_meas is not None else None, int(n_samples), int(jitter_seed))


# ---------------------------------------------------------------------------- entry points
def train_step(field, geom, view, pix, a_meas, n_samples, loss_out, ws, stream=None, jitter_seed=0):
    b = _batch(view, pix, a_meas, n_samples, jitter_seed)
    _check(load().train_step(field.handle, geom.handle, C.byref(b), _ptr(loss_out), _ptr(ws),
                             ws.numel() * 4, _stream(stream)), "train_step")


def accumulate_step(field, geom, view, pix, a_meas, n_samples, loss_out, ws, stream=None, jitter_seed=0):
    """Forward + loss + backward into the field's gradients, no optimizer step."""
    b = _batch(view, pix, a_meas, n_samples, jitter_seed)
    _check(load().accumulate_step(field.handle, geom.handle, C.byref(b), _ptr(loss_out), _ptr(ws),
                                  ws.numel() * 4, _stream(stream)), "accumulate_step")


def train_step_host(field, geom, view, pix_host, a_meas_host, n_samples, loss_host, ws, stream=None):
    """pix_host (int32), a_meas_host (float32), loss_host (float32[1]): CPU tensors, ideally pinned."""
    for t, dt in ((pix_host, torch.int32), (a_meas_host, torch.float32), (loss_host, torch.float32)):
        if t.is_cuda or t.dtype != dt or not t.is_contiguous():
            raise ValueError("train_step_host: expected contiguous host tensors")
    _check(load().train_step_host(field.handle, geom.handle, int(view), pix_host.numel(), _ptr(pix_host),
                                  _ptr(a_meas_host), int(n_samples), _ptr(loss_host), _ptr(ws),
                                  ws.numel() * 4, _stream(stream)), "train_step_host")


def render_forward(field, geom, view, pix, n_samples, a_pred, ws, stream=None, jitter_seed=0):
    b = _batch(view, pix, None, n_samples, jitter_seed)
    _check(load().render_forward(field.handle, geom.handle, C.byref(b), _ptr(a_pred), _ptr(ws),
                                 ws.numel() * 4, _stream(stream)), "render_forward")


def render_forward_noalloc(field, geom, view, pix, n_samples, a_pred, stream=None, jitter_seed=0):
    """render_forward without a workspace argument, for callers that cannot allocate
    device memory at call time; its scratch is a fixed 1 MiB block inside the library
    (see include/nhcbct.h for the size limit and the rules on concurrent calls)."""
    b = _batch(view, pix, None, n_samples, jitter_seed)
    _check(load().render_forward_noalloc(field.handle, geom.handle, C.byref(b), _ptr(a_pred), _stream(stream)),
           "render_forward_noalloc")


def render_backward(field, geom, view, pix, n_samples, dLdA, ws, stream=None, jitter_seed=0):
    b = _batch(view, pix, None, n_samples, jitter_seed)
    _check(load().render_backward(field.handle, geom.handle, C.byref(b), _ptr(dLdA), _ptr(ws),
                                  ws.numel() * 4, _stream(stream)), "render_backward")


def optimizer_step(field, stream=None):
    _check(load().optimizer_step(field.handle, _stream(stream)), "optimizer_step")


def fit_points_step(field, xyz, mu_gt, loss_out, ws, stream=None):
    xyz = _dev(xyz, torch.float32, "xyz")
    mu_gt = _dev(mu_gt, torch.float32, "mu_gt")
    _check(load().fit_points_step(field.handle, mu_gt.numel(), _ptr(xyz), _ptr(mu_gt), _ptr(loss_out),
                                  _ptr(ws), ws.numel() * 4, _stream(stream)), "fit_points_step")


def fit_points_backward(field, xyz, mu_gt, loss_out, ws, stream=None):
    xyz = _dev(xyz, torch.float32, "xyz")
    mu_gt = _dev(mu_gt, torch.float32, "mu_gt")
    _check(load().fit_points_backward(field.handle, mu_gt.numel(), _ptr(xyz), _ptr(mu_gt), _ptr(loss_out),
                                      _ptr(ws), ws.numel() * 4, _stream(stream)), "fit_points_backward")


def query_points(field, xyz, mu_out, stream=None):
    xyz = _dev(xyz, torch.float32, "xyz")
    _check(load().query_points(field.handle, mu_out.numel(), _ptr(xyz), _ptr(mu_out), _stream(stream)),
           "query_points")


def query_volume(field, D, out, stream=None):
    _check(load().query_volume(field.handle, int(D), _ptr(out), _stream(stream)), "query_volume")


def project(geom, vol, oversample, proj_out, stream=None):
    """vol: (D, D, D) or flat D^3 float32 CUDA tensor in [z][y][x] order."""
    vol = _dev(vol, torch.float32, "vol")
    D = vol.shape[0] if vol.dim() == 3 else int(round(vol.numel() ** (1.0 / 3.0)))
    if D ** 3 != vol.numel():
        raise ValueError("project: vol must hold D^3 voxels")
    _check(load().project(geom.handle, _ptr(vol), D, int(oversample), _ptr(proj_out),
                          _stream(stream)), "project")


def volume_mse(a, b, out=None, stream=None):
    """Device mean squared difference (float64 scalar tensor) of two float32 arrays."""
    a = _dev(a, torch.float32, "a")
    b = _dev(b, torch.float32, "b")
    if a.numel() != b.numel():
        raise ValueError("volume_mse: size mismatch")
    out = torch.empty(1, dtype=torch.float64, device=a.device) if out is None else out
    ws = torch.empty(1024, dtype=torch.float64, device=a.device)
    _check(load().volume_mse(_ptr(a), _ptr(b), a.numel(), _ptr(out), _ptr(ws), 8192, _stream(stream)),
           "volume_mse")
    return out


def ssim3d_workspace_bytes(D):
    out = _SZ()
    _check(load().ssim3d_workspace_bytes(int(D), C.byref(out)), "ssim3d_workspace_bytes")
    return out.value


def ssim3d(x, y, data_range=1.0, out=None, map_out=None, stream=None):
    """3-D SSIM (Sec. 3.2; Wang et al. 2004 settings) of two D^3 float32 CUDA volumes
    ([z][y][x]): returns the mean local index as a float64 device tensor of one
    element; map_out (float64, (D - 10)^3) receives the local index if given."""
    x = _dev(x, torch.float32, "x")
    y = _dev(y, torch.float32, "y")
    D = x.shape[0] if x.dim() == 3 else int(round(x.numel() ** (1.0 / 3.0)))
    if D ** 3 != x.numel() or y.numel() != x.numel():
        raise ValueError("ssim3d: x and y must both hold D^3 voxels")
    if map_out is not None:
        map_out = _dev(map_out, torch.float64, "map_out")
        if map_out.numel() != (D - 10) ** 3:
            raise ValueError("ssim3d: map_out must hold (D - 10)^3 values")
    out = torch.empty(1, dtype=torch.float64, device=x.device) if out is None else out
    nb = ssim3d_workspace_bytes(D)
    ws = torch.empty((nb + 7) // 8, dtype=torch.float64, device=x.device)
    _check(load().ssim3d(_ptr(x), _ptr(y), D, float(data_range), _ptr(out),
                         _ptr(map_out) if map_out is not None else None, _ptr(ws), nb, _stream(stream)), "ssim3d")
    return out


def ssim(vol_pred, vol_gt, data_range=1.0, stream=None):
    """Reconstruction SSIM (Sec. 3.2) of two D^3 volumes, a Python float."""
    return float(ssim3d(vol_pred, vol_gt, data_range, stream=stream).item())


def launch_info():
    """Grid decision of the last training-kernel launch (see include/nhcbct.h)."""
    out = (C.c_int32 * 6)()
    _check(load().launch_info(out, 6), "launch_info")
    keys = ("sms", "ctas_per_sm_occupancy", "ctas_per_sm_tmem", "grid", "tmem_cols", "smem_bytes")
    return dict(zip(keys, list(out)))


def psnr(vol_pred, vol_gt, data_range=1.0, stream=None):
    """Reconstruction PSNR (Sec. 3.2) in dB: 10 log10(range^2 / mse), mse from the library."""
    import math
    mse = float(volume_mse(vol_pred, vol_gt, stream=stream).item())
    return float("inf") if mse == 0 else 10.0 * math.log10(data_range * data_range / mse)


def sample_rays(geom, view, pix, n_samples, xyz_out, delta_out, stream=None, jitter_seed=0):
    pix = _dev(pix, torch.int32, "pix")
    _check(load().sample_rays(geom.handle, int(view), pix.numel(), _ptr(pix), int(n_samples), int(jitter_seed),
                              _ptr(xyz_out), _ptr(delta_out), _stream(stream)), "sample_rays")


def hash_corners(field, xyz, idx_out, w_out, stream=None):
    xyz = _dev(xyz, torch.float32, "xyz")
    _check(load().hash_corners(field.handle, xyz.numel() // 3, _ptr(xyz), _ptr(idx_out), _ptr(w_out),
                               _stream(stream)), "hash_corners")


def encode_points(field, xyz, h_out, stream=None):
    xyz = _dev(xyz, torch.float32, "xyz")
    _check(load().encode_points(field.handle, xyz.numel() // 3, _ptr(xyz), _ptr(h_out), _stream(stream)),
           "encode_points")


def channel_mask_workspace_bytes(field, G: int) -> int:
    out = C.c_size_t()
    _check(load().channel_mask_workspace_bytes(field.handle, G, C.byref(out)), "channel_mask_workspace_bytes")
    return out.value


def select_channel_mask(field, G, cutoff, threshold, apply, frac_out, mask_out, ws, stream=None):
    """FFT channel-mask selection in the library (include/nhcbct.h): frac_out float64
    [L F] and mask_out float32 [L F] (or None) on the device; apply installs the mask."""
    _check(load().field_select_channel_mask(field.handle, G, float(cutoff), float(threshold), int(bool(apply)),
                                            _ptr(frac_out), _ptr(mask_out), _ptr(ws), ws.numel() * 4,
                                            _stream(stream)), "field_select_channel_mask")


def scatter_points(field, xyz, dh, stream=None):
    """Adds the trilinear scatter of dh (float[n][L F]) at xyz into field.grads."""
    xyz = _dev(xyz, torch.float32, "xyz")
    dh = _dev(dh, torch.float32, "dh")
    _check(load().scatter_points(field.handle, xyz.numel() // 3, _ptr(xyz), _ptr(dh), _stream(stream)),
           "scatter_points")


# ---------------------------------------------------------------------------- roofline probes
def probe_l2_read(buf, reps, sink, stream=None):
    _check(load().probe_l2_read(_ptr(buf), buf.numel() * buf.element_size(), int(reps), _ptr(sink),
                                _stream(stream)), "probe_l2_read")


def probe_random_gather(table, entry_bytes, n_loads, sink, stream=None):
    """Random entry_bytes loads from table (n_entries = bytes / entry_bytes); returns the count issued."""
    done = C.c_int64()
    n_entries = table.numel() * table.element_size() // entry_bytes
    _check(load().probe_random_gather(_ptr(table), n_entries, int(entry_bytes), int(n_loads), _ptr(sink),
                                      C.byref(done), _stream(stream)), "probe_random_gather")
    return done.value


def probe_random_red(table, n_ops, stream=None):
    """Random float2 atomic adds into table (float32, even length); returns the count issued."""
    done = C.c_int64()
    _check(load().probe_random_red(_ptr(table), table.numel() // 2, int(n_ops), C.byref(done), _stream(stream)),
           "probe_random_red")
    return done.value


def probe_random_red16(table, fmt, n_ops, stream=None):
    """Random packed 16-bit atomic adds (fmt PREC_BF16 or PREC_F16) into the 4-byte
    entries of table (any dtype, 4-byte aligned); returns the count issued."""
    done = C.c_int64()
    n_entries = table.numel() * table.element_size() // 4
    _check(load().probe_random_red16(_ptr(table), n_entries, int(fmt), int(n_ops), C.byref(done),
                                     _stream(stream)), "probe_random_red16")
    return done.value


# ---------------------------------------------------------------------------- autograd
class Render(torch.autograd.Function):
    """A = render(params) through the hand-written CUDA forward and backward.

    ``params`` is the field's flat parameter tensor; the backward recomputes the
    features on the GPU and returns dL/dparams (gradients are not accumulated into
    the field's optimizer buffers)."""

    @staticmethod
    def forward(ctx, params, field, geom, view, pix, n_samples):
        ws = workspace(step_workspace_bytes(field, pix.numel(), n_samples), params.device)
        a = torch.empty(pix.numel(), dtype=torch.float32, device=params.device)
        render_forward(field, geom, view, pix, n_samples, a, ws)
        ctx.save_for_backward(pix)
        ctx.field, ctx.geom, ctx.view, ctx.n = field, geom, view, n_samples
        return a

    @staticmethod
    def backward(ctx, dA):
        (pix,) = ctx.saved_tensors
        f = ctx.field
        saved = f.grads.clone()
        f.grads.zero_()
        ws = workspace(step_workspace_bytes(f, pix.numel(), ctx.n), dA.device)
        render_backward(f, ctx.geom, ctx.view, pix, ctx.n, dA.contiguous().float(), ws)
        _, scale, _ = f.poll_status()
        g = f.grads[: f.n_params].clone() / scale
        f.grads.copy_(saved)
        return g, None, None, None, None, None
