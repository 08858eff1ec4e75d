"""ctypes binding of libsgsplat.so: the C ABI declared in include/sgsplat.h.

Argument marshalling only. Every step of the rasterizer runs in the CUDA
library; there is no CPU fallback. If the library has not been built, or no
CUDA device is present, calls raise instead of computing anything.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np
import torch

from . import build as _build

SG_OK, SG_ERR_INVALID_ARG, SG_ERR_WORKSPACE, SG_ERR_CAPACITY, SG_ERR_TIMEOUT, SG_ERR_CUDA = range(6)
SG_F32, SG_F16, SG_BF16 = 0, 1, 2
SG_COLOR_SG, SG_COLOR_SH3 = 0, 1
SG_MAX_VIEWS = 128
SG_MAX_SCENES = 32

STATUS_NAMES = {0: "SG_OK", 1: "SG_ERR_INVALID_ARG", 2: "SG_ERR_WORKSPACE", 3: "SG_ERR_CAPACITY",
                4: "SG_ERR_TIMEOUT", 5: "SG_ERR_CUDA"}

EXPORTS = ("sg_version", "sg_last_error", "sg_workspace_query", "sg_workspace_layout",
           "sg_render_forward", "sg_render_backward", "sg_profile_enable", "sg_profile_read",
           "sg_profile_stage_name", "sg_kernel_launches", "sg_render_backward_noalloc",
           "sg_set_tuning", "sg_get_tuning", "sg_batched_workspace_query",
           "sg_render_batched_forward", "sg_render_batched_backward", "sg_forward_status",
           "sg_batched_workspace_layout",
           "sg_render_forward_importance", "sg_admm_workspace_bytes", "sg_admm_opacity_step",
           "sg_admm_sharpness_step", "sg_admm_penalty_grad", "sg_postprocess_workspace_bytes",
           "sg_postprocess_plan", "sg_postprocess_apply")
SG_NOALLOC_SCRATCH_BYTES = 16 << 20
SG_PROFILE_EVENTS, SG_PROFILE_COUNT, SG_PROFILE_STAGES = 1, 2, 12

_P = ctypes.c_void_p


class sg_scene(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("n_lobes", ctypes.c_int64),
                ("dtype_geom", ctypes.c_int32), ("dtype_lobe", ctypes.c_int32),
                ("dtype_sharp", ctypes.c_int32), ("color_model", ctypes.c_int32),
                ("means", _P), ("scales", _P), ("quats", _P), ("opac", _P), ("gmask", _P),
                ("c0", _P), ("lobe_off", _P), ("axis", _P), ("sharp", _P), ("amp", _P),
                ("lmask", _P), ("sh", _P)]


class sg_camera(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("fx", ctypes.c_float), ("fy", ctypes.c_float), ("cx", ctypes.c_float),
                ("cy", ctypes.c_float), ("viewmat", ctypes.c_float * 12),
                ("near_plane", ctypes.c_float), ("bg", ctypes.c_float * 3)]


class sg_grads(ctypes.Structure):
    _fields_ = [(k, _P) for k in ("means", "scales", "quats", "opac", "gmask", "c0", "axis",
                                  "sharp", "amp", "lmask", "sh")]


class sg_sizes(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint64) for k in (
        "n_entries", "n_tiles", "n_pixels", "n_pairs", "pair_capacity", "ws_fixed_bytes",
        "ws_per_pair_bytes", "ws_bytes", "bwd_ws_bytes")]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class sg_ws_layout(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint64) for k in (
        "rec", "tiles_touched", "rect", "depth_order", "ranges", "pair_tile", "pair_entry",
        "total_bytes")]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class sg_tuning(ctypes.Structure):
    _fields_ = [("fwd_pixels_per_thread", ctypes.c_int32), ("bwd_pixels_per_thread", ctypes.c_int32),
                ("fwd_persistent", ctypes.c_int32), ("bwd_persistent", ctypes.c_int32),
                ("sort_wait_polls", ctypes.c_int32), ("fwd_batch", ctypes.c_int32),
                ("bwd_batch", ctypes.c_int32), ("reserved", ctypes.c_int32 * 1)]


TUNING_FIELDS = ("fwd_pixels_per_thread", "bwd_pixels_per_thread", "fwd_persistent", "bwd_persistent",
                 "sort_wait_polls", "fwd_batch", "bwd_batch")


class SGError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_LIB = None


def library_path():
    return _build.library_path()


def lib():
    """Loads libsgsplat.so (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"libsgsplat.so not built ({path}); run "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(path)
        L.sg_version.argtypes = []
        L.sg_version.restype = ctypes.c_int
        L.sg_last_error.argtypes = []
        L.sg_last_error.restype = ctypes.c_char_p
        L.sg_workspace_query.argtypes = [ctypes.POINTER(sg_scene), ctypes.POINTER(sg_camera),
                                         ctypes.c_int, ctypes.c_uint64, ctypes.POINTER(sg_sizes)]
        L.sg_workspace_query.restype = ctypes.c_int
        L.sg_workspace_layout.argtypes = [ctypes.POINTER(sg_scene), ctypes.POINTER(sg_camera),
                                          ctypes.c_int, ctypes.c_size_t, ctypes.POINTER(sg_ws_layout)]
        L.sg_workspace_layout.restype = ctypes.c_int
        L.sg_render_forward.argtypes = [ctypes.POINTER(sg_scene), ctypes.POINTER(sg_camera),
                                        ctypes.c_int, _P, ctypes.c_size_t, _P, _P, _P,
                                        ctypes.POINTER(sg_sizes), _P]
        L.sg_render_forward.restype = ctypes.c_int
        L.sg_render_backward.argtypes = [ctypes.POINTER(sg_scene), ctypes.POINTER(sg_camera),
                                         ctypes.c_int, _P, ctypes.c_size_t, _P, _P, _P, _P,
                                         ctypes.c_size_t, ctypes.POINTER(sg_grads), _P]
        L.sg_render_backward.restype = ctypes.c_int
        L.sg_autotune.argtypes = [ctypes.POINTER(sg_scene), ctypes.POINTER(sg_camera), ctypes.c_int,
                                  _P, ctypes.c_size_t, _P, _P, _P, _P, _P, ctypes.c_size_t,
                                  ctypes.POINTER(sg_grads), ctypes.c_int, ctypes.POINTER(sg_tuning), _P, _P]
        L.sg_autotune.restype = ctypes.c_int
        L.sg_profile_enable.argtypes = [ctypes.c_int]
        L.sg_profile_enable.restype = ctypes.c_int
        L.sg_profile_set_stages.argtypes = [ctypes.c_uint32]
        L.sg_profile_set_stages.restype = ctypes.c_int
        L.sg_profile_read.argtypes = [_P, _P, _P, ctypes.c_int]
        L.sg_profile_read.restype = ctypes.c_int
        L.sg_render_backward_noalloc.argtypes = [ctypes.POINTER(sg_scene), ctypes.POINTER(sg_camera),
                                                 ctypes.c_int, _P, ctypes.c_size_t, _P, _P, _P,
                                                 ctypes.POINTER(sg_grads), _P]
        L.sg_render_backward_noalloc.restype = ctypes.c_int
        L.sg_set_tuning.argtypes = [ctypes.POINTER(sg_tuning)]
        L.sg_set_tuning.restype = ctypes.c_int
        L.sg_get_tuning.argtypes = [ctypes.POINTER(sg_tuning)]
        L.sg_get_tuning.restype = ctypes.c_int
        PS, PC = ctypes.POINTER(sg_scene), ctypes.POINTER(sg_camera)
        L.sg_batched_workspace_query.argtypes = [PS, ctypes.c_int, PC, _P, ctypes.c_int, ctypes.c_uint64,
                                                 ctypes.POINTER(sg_sizes)]
        L.sg_batched_workspace_query.restype = ctypes.c_int
        L.sg_batched_workspace_layout.argtypes = [PS, ctypes.c_int, PC, _P, ctypes.c_int, ctypes.c_size_t,
                                                  ctypes.POINTER(sg_ws_layout)]
        L.sg_batched_workspace_layout.restype = ctypes.c_int
        L.sg_render_batched_forward.argtypes = [PS, ctypes.c_int, PC, _P, ctypes.c_int, _P, ctypes.c_size_t,
                                                _P, _P, _P, _P, _P]
        L.sg_render_forward_importance.argtypes = [PS, PC, ctypes.c_int, _P, ctypes.c_size_t, _P, _P, _P,
                                                   _P, ctypes.POINTER(sg_sizes), _P]
        L.sg_render_forward_importance.restype = ctypes.c_int
        L.sg_render_batched_forward.restype = ctypes.c_int
        L.sg_render_batched_backward.argtypes = [PS, ctypes.c_int, PC, _P, ctypes.c_int, _P, ctypes.c_size_t,
                                                 _P, _P, _P, _P, ctypes.c_size_t, ctypes.POINTER(sg_grads), _P]
        L.sg_render_batched_backward.restype = ctypes.c_int
        L.sg_forward_status.argtypes = [_P, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_int32), _P]
        L.sg_forward_status.restype = ctypes.c_int
        L.sg_admm_workspace_bytes.argtypes = [ctypes.c_int64]
        L.sg_admm_workspace_bytes.restype = ctypes.c_size_t
        L.sg_admm_opacity_step.argtypes = [ctypes.c_int64, _P, _P, ctypes.c_int64, _P, _P, _P,
                                           ctypes.c_size_t, _P]
        L.sg_admm_opacity_step.restype = ctypes.c_int
        L.sg_admm_sharpness_step.argtypes = [ctypes.c_int64, _P, _P, ctypes.c_int64, _P, _P, _P,
                                             ctypes.c_size_t, _P]
        L.sg_admm_sharpness_step.restype = ctypes.c_int
        L.sg_admm_penalty_grad.argtypes = [ctypes.c_int64, _P, _P, _P, ctypes.c_float, _P, _P]
        L.sg_admm_penalty_grad.restype = ctypes.c_int
        L.sg_postprocess_workspace_bytes.argtypes = [ctypes.c_int64]
        L.sg_postprocess_workspace_bytes.restype = ctypes.c_size_t
        L.sg_postprocess_plan.argtypes = [PS, ctypes.c_float, ctypes.c_float, _P, ctypes.c_size_t,
                                          ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64), _P]
        L.sg_postprocess_plan.restype = ctypes.c_int
        L.sg_postprocess_apply.argtypes = [PS, ctypes.c_float, ctypes.c_float, _P, ctypes.c_size_t, PS, _P]
        L.sg_postprocess_apply.restype = ctypes.c_int
        L.sg_kernel_launches.argtypes = []
        L.sg_kernel_launches.restype = ctypes.c_int64
        L.sg_profile_stage_name.argtypes = [ctypes.c_int]
        L.sg_profile_stage_name.restype = ctypes.c_char_p
        _LIB = L
    return _LIB


def _check(status):
    if status != SG_OK:
        raise SGError(status, lib().sg_last_error().decode())
    return status


def _ptr(t):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _stream_handle(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


# ---------------------------------------------------------------------------
# Host-side descriptions
# ---------------------------------------------------------------------------

_TORCH_DT = {SG_F32: torch.float32, SG_F16: torch.float16, SG_BF16: torch.bfloat16}


@dataclass
class DeviceScene:
    """Scene arrays on the GPU in the planar layout of sg_scene."""
    means: torch.Tensor
    scales: torch.Tensor
    quats: torch.Tensor
    opac: torch.Tensor
    gmask: torch.Tensor
    c0: torch.Tensor
    lobe_off: torch.Tensor
    axis: torch.Tensor
    sharp: torch.Tensor
    amp: torch.Tensor
    lmask: torch.Tensor
    dtype_geom: int = SG_F32
    dtype_lobe: int = SG_F32
    dtype_sharp: int = SG_F32
    sh: torch.Tensor | None = None   # [3][16][N] SH3 coefficients: the SH colour model

    @property
    def color_model(self):
        return SG_COLOR_SH3 if self.sh is not None else SG_COLOR_SG

    def grad_fields(self):
        return self.FLOAT_FIELDS + (("sh",) if self.sh is not None else ())

    FLOAT_FIELDS = ("means", "scales", "quats", "opac", "gmask", "c0", "axis", "sharp", "amp",
                    "lmask")

    @property
    def n(self):
        return int(self.means.shape[1])

    @property
    def n_lobes(self):
        return int(self.sharp.shape[0])

    @classmethod
    def from_host(cls, scene, device="cuda", storage="f32"):
        """storage: 'f32' | 'f16' (geometry and lobes in binary16) | 'f16_bf16s'
        (as f16, sharpness in bfloat16)."""
        dg, dl, ds = {"f32": (SG_F32,) * 3, "f16": (SG_F16,) * 3,
                      "f16_bf16s": (SG_F16, SG_F16, SG_BF16)}[storage]
        fam = {"means": dg, "scales": dg, "quats": dg, "opac": dg, "axis": dl, "amp": dl,
               "sharp": ds}
        kw = {}
        for k in cls.FLOAT_FIELDS:
            a = torch.from_numpy(np.ascontiguousarray(getattr(scene, k), np.float32))
            kw[k] = a.to(device=device, dtype=_TORCH_DT[fam.get(k, SG_F32)]).contiguous()
        kw["lobe_off"] = torch.from_numpy(np.ascontiguousarray(scene.lobe_off, np.int32)).to(device)
        if getattr(scene, "sh", None) is not None:
            kw["sh"] = torch.from_numpy(np.ascontiguousarray(scene.sh, np.float32)).to(device)
        return cls(dtype_geom=dg, dtype_lobe=dl, dtype_sharp=ds, **kw)

    def struct(self):
        s = sg_scene()
        s.n = self.n
        s.n_lobes = self.n_lobes
        s.dtype_geom, s.dtype_lobe, s.dtype_sharp = self.dtype_geom, self.dtype_lobe, self.dtype_sharp
        s.color_model = self.color_model
        for k in self.FLOAT_FIELDS + ("lobe_off",):
            t = getattr(self, k)
            setattr(s, k, t.data_ptr() if t.numel() else None)
        s.sh = self.sh.data_ptr() if self.sh is not None and self.sh.numel() else None
        return s


def camera_struct(cam):
    c = sg_camera()
    c.width, c.height = int(cam.width), int(cam.height)
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    vm = np.asarray(cam.viewmat, np.float32).reshape(12)
    for i in range(12):
        c.viewmat[i] = float(vm[i])
    c.near_plane = float(cam.near)
    bg = np.asarray(cam.bg, np.float32).reshape(3)
    for i in range(3):
        c.bg[i] = float(bg[i])
    return c


def camera_array(cams):
    arr = (sg_camera * len(cams))()
    for i, cam in enumerate(cams):
        arr[i] = camera_struct(cam)
    return arr


def grads_struct(grads: dict):
    g = sg_grads()
    for k, _ in sg_grads._fields_:
        t = grads.get(k)
        setattr(g, k, t.data_ptr() if (t is not None and t.numel()) else None)
    return g


# ---------------------------------------------------------------------------
# The C entry points, same names
# ---------------------------------------------------------------------------

def sg_version() -> int:
    return int(lib().sg_version())


def sg_last_error() -> str:
    return lib().sg_last_error().decode()


def sg_workspace_query(scene: DeviceScene, cams, pair_capacity: int) -> dict:
    s = scene.struct()
    c = camera_array(cams)
    out = sg_sizes()
    _check(lib().sg_workspace_query(ctypes.byref(s), c, len(cams), int(pair_capacity),
                                    ctypes.byref(out)))
    return out.as_dict()


NO_OFFSET = 2**64 - 1   # a layout entry for a buffer the workspace does not hold


def sg_workspace_layout(scene: DeviceScene, cams, ws_bytes: int) -> dict:
    """Byte offsets of a forward's buffers in a workspace of ws_bytes. pair_tile
    is NO_OFFSET when the views have at most 12288 tiles in all: the tile sort
    then counts and keeps no sorted tile ids (pair k's tile is the tile whose
    range holds k)."""
    s = scene.struct()
    c = camera_array(cams)
    out = sg_ws_layout()
    _check(lib().sg_workspace_layout(ctypes.byref(s), c, len(cams), int(ws_bytes), ctypes.byref(out)))
    return out.as_dict()


def sg_render_forward(scene: DeviceScene, cams, ws: torch.Tensor, img, T_final, last,
                      stream=None, raise_on_error=True):
    """Returns (status, sizes dict). Raises SGError on failure unless
    raise_on_error is False (then the status is returned)."""
    s = scene.struct()
    c = camera_array(cams)
    out = sg_sizes()
    st = lib().sg_render_forward(ctypes.byref(s), c, len(cams), _ptr(ws), ws.numel(), _ptr(img),
                                 _ptr(T_final), _ptr(last), ctypes.byref(out),
                                 _stream_handle(stream))
    if raise_on_error:
        _check(st)
    return st, out.as_dict()


def sg_render_backward(scene: DeviceScene, cams, ws, T_final, last, d_img, bwd_ws, grads: dict,
                       stream=None):
    s = scene.struct()
    c = camera_array(cams)
    g = grads_struct(grads)
    _check(lib().sg_render_backward(ctypes.byref(s), c, len(cams), _ptr(ws), ws.numel(),
                                    _ptr(T_final), _ptr(last), _ptr(d_img), _ptr(bwd_ws),
                                    bwd_ws.numel(), ctypes.byref(g), _stream_handle(stream)))


def sg_autotune(scene: DeviceScene, cams, ws, img, T_final, last, d_img, bwd_ws, grads: dict, reps=3,
                stream=None) -> dict:
    """Times every blend shape on this workload and installs the fastest (see
    sgsplat.h). Returns the choice and the per-candidate mean times (ms)."""
    s = scene.struct()
    c = camera_array(cams)
    g = grads_struct(grads)
    t = sg_tuning()
    times = (ctypes.c_float * 16)()
    _check(lib().sg_autotune(ctypes.byref(s), c, len(cams), _ptr(ws), ws.numel(), _ptr(img), _ptr(T_final),
                             _ptr(last), _ptr(d_img), _ptr(bwd_ws), bwd_ws.numel(), ctypes.byref(g),
                             int(reps), ctypes.byref(t), ctypes.cast(times, _P), _stream_handle(stream)))
    names = [f"p{1 << (k >> 1)}" + ("_persistent" if k & 1 else "") for k in range(8)]
    return {"fwd_pixels_per_thread": t.fwd_pixels_per_thread, "bwd_pixels_per_thread": t.bwd_pixels_per_thread,
            "fwd_persistent": t.fwd_persistent, "bwd_persistent": t.bwd_persistent,
            "fwd_batch": t.fwd_batch, "bwd_batch": t.bwd_batch,
            "ms": {names[k]: {"fwd_call": times[k], "bwd_call": times[8 + k]} for k in range(8)}}


def sg_profile_enable(flags: int):
    _check(lib().sg_profile_enable(int(flags)))


def sg_profile_set_stages(stage_mask: int):
    """Bit i: stage i is bracketed by events when SG_PROFILE_EVENTS is on (default all)."""
    _check(lib().sg_profile_set_stages(ctypes.c_uint32(stage_mask & 0xFFFFFFFF)))


def sg_profile_stage_name(i: int):
    r = lib().sg_profile_stage_name(int(i))
    return None if r is None else r.decode()


def sg_profile_read(reset=True) -> dict:
    """Per-stage GPU milliseconds and launch counts since the last reset, plus
    pair evaluations of the counting blend kernels."""
    ms = (ctypes.c_double * SG_PROFILE_STAGES)()
    n = (ctypes.c_int64 * SG_PROFILE_STAGES)()
    ev = (ctypes.c_int64 * 2)()
    _check(lib().sg_profile_read(ctypes.cast(ms, _P), ctypes.cast(n, _P), ctypes.cast(ev, _P),
                                 int(bool(reset))))
    stages = {sg_profile_stage_name(i): {"ms": ms[i], "launches": int(n[i])}
              for i in range(SG_PROFILE_STAGES)}
    return {"stages": stages, "pair_evals": {"forward": int(ev[0]), "backward": int(ev[1])}}


def sg_kernel_launches() -> int:
    return int(lib().sg_kernel_launches())


def sg_render_backward_noalloc(scene: DeviceScene, cams, ws, T_final, last, d_img, grads: dict,
                               stream=None, raise_on_error=True):
    """Backward whose scratch is the library's static device array (for callers
    that cannot allocate device memory while rendering). Returns the status."""
    s = scene.struct()
    c = camera_array(cams)
    g = grads_struct(grads)
    st = lib().sg_render_backward_noalloc(ctypes.byref(s), c, len(cams), _ptr(ws), ws.numel(),
                                          _ptr(T_final), _ptr(last), _ptr(d_img), ctypes.byref(g),
                                          _stream_handle(stream))
    if raise_on_error:
        _check(st)
    return st


def sg_set_tuning(fwd_pixels_per_thread=None, bwd_pixels_per_thread=None, fwd_persistent=None,
                  bwd_persistent=None, sort_wait_polls=None, fwd_batch=None, bwd_batch=None):
    """Sets the kernels' tuning (unset fields keep their value); no arguments
    restores the defaults."""
    args = (fwd_pixels_per_thread, bwd_pixels_per_thread, fwd_persistent, bwd_persistent, sort_wait_polls,
            fwd_batch, bwd_batch)
    if all(a is None for a in args):
        _check(lib().sg_set_tuning(None))
        return
    cur = sg_get_tuning()
    t = sg_tuning()
    for name, val in zip(TUNING_FIELDS, args):
        setattr(t, name, int(cur[name] if val is None else val))
    _check(lib().sg_set_tuning(ctypes.byref(t)))


def sg_get_tuning() -> dict:
    t = sg_tuning()
    _check(lib().sg_get_tuning(ctypes.byref(t)))
    return {k: int(getattr(t, k)) for k in TUNING_FIELDS}


# ---------------------------------------------------------------------------
# batched form
# ---------------------------------------------------------------------------

def scene_array(scenes):
    arr = (sg_scene * len(scenes))()
    for i, sc in enumerate(scenes):
        arr[i] = sc.struct()
    return arr


def _view_scene_array(view_scene):
    return (ctypes.c_int32 * len(view_scene))(*[int(v) for v in view_scene])


def sg_batched_workspace_query(scenes, cams, view_scene, pair_capacity: int) -> dict:
    out = sg_sizes()
    _check(lib().sg_batched_workspace_query(scene_array(scenes), len(scenes), camera_array(cams),
                                            _view_scene_array(view_scene), len(cams),
                                            int(pair_capacity), ctypes.byref(out)))
    return out.as_dict()


def sg_batched_workspace_layout(scenes, cams, view_scene, ws_bytes: int) -> dict:
    """As sg_workspace_layout, for a batched forward."""
    out = sg_ws_layout()
    _check(lib().sg_batched_workspace_layout(scene_array(scenes), len(scenes), camera_array(cams),
                                             _view_scene_array(view_scene), len(cams), int(ws_bytes),
                                             ctypes.byref(out)))
    return out.as_dict()


def sg_render_batched_forward(scenes, cams, view_scene, ws, img, T_final, last, importance=None,
                              stream=None):
    imp = None
    if importance is not None:
        imp = (ctypes.c_void_p * len(scenes))(*[t.data_ptr() if t.numel() else None for t in importance])
    _check(lib().sg_render_batched_forward(scene_array(scenes), len(scenes), camera_array(cams),
                                           _view_scene_array(view_scene), len(cams), _ptr(ws),
                                           ws.numel(), _ptr(img), _ptr(T_final), _ptr(last),
                                           imp, _stream_handle(stream)))


def sg_render_forward_importance(scene: DeviceScene, cams, ws, img, T_final, last, importance,
                                 stream=None, raise_on_error=True):
    s = scene.struct()
    c = camera_array(cams)
    out = sg_sizes()
    st = lib().sg_render_forward_importance(ctypes.byref(s), c, len(cams), _ptr(ws), ws.numel(),
                                            _ptr(img), _ptr(T_final), _ptr(last), _ptr(importance),
                                            ctypes.byref(out), _stream_handle(stream))
    if raise_on_error:
        _check(st)
    return st, out.as_dict()


def sg_render_batched_backward(scenes, cams, view_scene, ws, T_final, last, d_img, bwd_ws,
                               grads_list, stream=None):
    g = (sg_grads * len(grads_list))()
    for i, gd in enumerate(grads_list):
        g[i] = grads_struct(gd)
    _check(lib().sg_render_batched_backward(scene_array(scenes), len(scenes), camera_array(cams),
                                            _view_scene_array(view_scene), len(cams), _ptr(ws),
                                            ws.numel(), _ptr(T_final), _ptr(last), _ptr(d_img),
                                            _ptr(bwd_ws), bwd_ws.numel(), g, _stream_handle(stream)))


def sg_forward_status(ws, stream=None):
    """(pairs needed by the last forward on ws, status). Synchronises the stream."""
    n = ctypes.c_uint64()
    st = ctypes.c_int32()
    _check(lib().sg_forward_status(_ptr(ws), ctypes.byref(n), ctypes.byref(st), _stream_handle(stream)))
    return int(n.value), int(st.value)


# ---------------------------------------------------------------------------
# ADMM steps (Alg. 1)
# ---------------------------------------------------------------------------

def sg_admm_workspace_bytes(n: int) -> int:
    return int(lib().sg_admm_workspace_bytes(int(n)))


def _admm_ws(n, ws, device):
    need = sg_admm_workspace_bytes(n)
    if ws is None or ws.numel() < need:
        ws = torch.empty(max(need, 256), dtype=torch.uint8, device=device)
    return ws


def sg_admm_opacity_step(opac, lam, opac_tilde, kappa, importance=None, ws=None, stream=None):
    """Proximal step (top-kappa by importance, or by |opac + lambda|) and dual
    update, in place on lam and opac_tilde."""
    n = opac.numel()
    ws = _admm_ws(n, ws, opac.device)
    _check(lib().sg_admm_opacity_step(n, _ptr(opac), _ptr(importance), int(kappa), _ptr(lam),
                                      _ptr(opac_tilde), _ptr(ws), ws.numel(), _stream_handle(stream)))
    return ws


def sg_admm_sharpness_step(sharp, amp, lam, sharp_tilde, kappa, ws=None, stream=None):
    """Proximal step (top-kappa lobes by dynamic range) and dual update."""
    n = sharp.numel()
    ws = _admm_ws(n, ws, sharp.device)
    _check(lib().sg_admm_sharpness_step(n, _ptr(sharp), _ptr(amp), int(kappa), _ptr(lam),
                                        _ptr(sharp_tilde), _ptr(ws), ws.numel(), _stream_handle(stream)))
    return ws


def sg_admm_penalty_grad(x, x_tilde, lam, delta, grad, stream=None):
    """grad += delta * (x - x_tilde + lam), in place."""
    _check(lib().sg_admm_penalty_grad(x.numel(), _ptr(x), _ptr(x_tilde), _ptr(lam), float(delta),
                                      _ptr(grad), _stream_handle(stream)))


# ---------------------------------------------------------------------------
# post-processing (Sec. 3.3.3)
# ---------------------------------------------------------------------------

def sg_postprocess(scene: DeviceScene, tau_opacity: float, tau_sharpness: float = 1.0,
                   stream=None) -> DeviceScene:
    """Removes low-opacity Gaussians and low-sharpness lobes (with the colour
    compensation of Eq. 12-13) and returns the compacted binary32 scene."""
    dev = scene.means.device
    n = scene.n
    ws = torch.empty(max(int(lib().sg_postprocess_workspace_bytes(n)), 256), dtype=torch.uint8,
                     device=dev)
    s_in = scene.struct()
    n_out, l_out = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().sg_postprocess_plan(ctypes.byref(s_in), float(tau_opacity), float(tau_sharpness),
                                     _ptr(ws), ws.numel(), ctypes.byref(n_out), ctypes.byref(l_out),
                                     _stream_handle(stream)))
    N, L = int(n_out.value), int(l_out.value)
    f = dict(device=dev, dtype=torch.float32)
    out = DeviceScene(means=torch.empty(3, N, **f), scales=torch.empty(3, N, **f),
                      quats=torch.empty(4, N, **f), opac=torch.empty(N, **f), gmask=torch.empty(N, **f),
                      c0=torch.empty(3, N, **f), lobe_off=torch.empty(N + 1, dtype=torch.int32, device=dev),
                      axis=torch.empty(3, L, **f), sharp=torch.empty(L, **f), amp=torch.empty(3, L, **f),
                      lmask=torch.empty(L, **f))
    s_out = out.struct()
    s_out.lobe_off = out.lobe_off.data_ptr()
    _check(lib().sg_postprocess_apply(ctypes.byref(s_in), float(tau_opacity), float(tau_sharpness),
                                      _ptr(ws), ws.numel(), ctypes.byref(s_out), _stream_handle(stream)))
    return out
