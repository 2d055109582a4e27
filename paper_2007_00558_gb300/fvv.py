"""Thin ctypes binding of libfvv.so (include/fvv.h): same names, argument
marshalling only.  Every step of view synthesis runs in the library's CUDA
kernels; there is no Python or CPU fallback, and loading fails loudly when the
library has not been built.

Pointers may be passed as ints, numpy arrays or torch tensors (host or CUDA);
``stream`` may be None, an int handle, or a torch.cuda.Stream.
"""
from __future__ import annotations

import ctypes as C
import os
import re
import threading
from typing import Optional, Sequence

import numpy as np

from . import build as _build

FVV_OK = 0
FVV_ERR_INVALID_ARG = 1
FVV_ERR_OUT_OF_MEMORY = 2
FVV_ERR_BUDGET = 3
FVV_ERR_CUDA = 4
FVV_ERR_TIMEOUT = 5
FVV_ERR_BUSY = 6
FVV_ERR_NOT_READY = 7
FVV_ERR_STATE = 8
FVV_MAX_CAMS = 64
FVV_MAX_SRC_PIXELS = 1 << 26
FVV_KEY_EMPTY = 0xFFFFFFFFFFFFFFFF
FVV_DEPTH_BG = 65535
FVV_NOALLOC_MAX_PIXELS = 1 << 21

_NAMES = {v: k for k, v in list(globals().items()) if k.startswith("FVV_ERR_") or k == "FVV_OK"}


class FvvError(RuntimeError):
    def __init__(self, code: int, func: str, msg: str):
        super().__init__("%s failed: %s (%s)" % (func, msg, _NAMES.get(code, code)))
        self.code = code


class fvv_camera(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32),
                ("fx", C.c_double), ("fy", C.c_double), ("cx", C.c_double), ("cy", C.c_double),
                ("R", C.c_double * 9), ("t", C.c_double * 3)]


fvv_view = fvv_camera


class fvv_rig(C.Structure):
    _fields_ = [("n_cams", C.c_int32), ("cams", C.POINTER(fvv_camera)),
                ("look_at", C.c_double * 3), ("depth_unit_m", C.c_double)]


class fvv_options(C.Structure):
    _fields_ = [("n_ref", C.c_int32), ("crack_filter", C.c_int32), ("hole_fill", C.c_int32),
                ("tau_crack", C.c_float), ("tau_vis", C.c_float), ("z_min", C.c_float),
                ("d_lo", C.c_uint32), ("d_hi", C.c_uint32), ("frame_slots", C.c_int32),
                ("max_batch", C.c_int32), ("memory_budget", C.c_uint64), ("layered", C.c_int32),
                ("jbf_radius", C.c_int32), ("jbf_sigma_s", C.c_float), ("jbf_sigma_c", C.c_float),
                ("jbf_min_valid", C.c_int32), ("pixel_weights", C.c_int32)]


class fvv_aux(C.Structure):
    _fields_ = [("depth", C.c_void_p), ("hole", C.c_void_p), ("top3", C.c_void_p),
                ("keys", C.c_void_p), ("keys_raw", C.c_void_p)]


class fvv_serve_cfg(C.Structure):
    _fields_ = [("lanes", C.c_int32), ("max_batch", C.c_int32), ("max_pending", C.c_int32),
                ("memory_budget", C.c_uint64), ("refine", C.c_int32), ("persistent", C.c_int32),
                ("max_width", C.c_int32), ("idle_us", C.c_uint32), ("batch_window_us", C.c_uint32)]


class fvv_serve_report(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64), ("failed", C.c_uint64),
                ("batches", C.c_uint64), ("mean_batch", C.c_double), ("p50_ms", C.c_double),
                ("p99_ms", C.c_double), ("max_ms", C.c_double), ("views_per_s", C.c_double),
                ("in_flight", C.c_int32)]


class fvv_unet_cfg(C.Structure):
    _fields_ = [("widths", C.c_int32 * 3), ("seed", C.c_uint64), ("z_far", C.c_float)]


class fvv_refine_batch(C.Structure):
    _fields_ = [("n", C.c_int32), ("height", C.c_int32), ("width", C.c_int32),
                ("rgb", C.c_void_p), ("depth", C.c_void_p), ("hole", C.c_void_p),
                ("top3", C.c_void_p), ("target", C.c_void_p)]


FVV_REFINE_PARAMS, FVV_REFINE_GRADS, FVV_REFINE_ADAM_M, FVV_REFINE_ADAM_V = 0, 1, 2, 3


class fvv_kernel_stats(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", C.c_uint64), ("timed", C.c_uint64),
                ("total_ms", C.c_double)]


_lib = None
_lock = threading.Lock()


def lib_path() -> str:
    return _build.LIB


def load() -> C.CDLL:
    """Load libfvv.so (built in-tree by ``paper_2007_00558_gb300.build``)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError("libfvv.so is not built (%s); run __graft_entry__.build() or "
                               "python -m paper_2007_00558_gb300.build" % path)
        lib = C.CDLL(path)
        P, S, I, U64 = C.c_void_p, C.c_size_t, C.c_int32, C.c_uint64
        sig = {
            "fvv_default_options": [C.POINTER(fvv_options)],
            "fvv_last_error": [],
            "fvv_create": [C.POINTER(fvv_rig), C.POINTER(fvv_options), C.POINTER(P)],
            "fvv_destroy": [P],
            "fvv_upload_frame": [P, I, P, S, P, S, U64, P],
            "fvv_upload_frames": [P, P, S, S, P, S, S, U64, P],
            "fvv_set_bg_depth": [P, I, P, S],
            "fvv_upload_frames_subset": [P, U64, P, S, S, P, S, S, U64, P],
            "fvv_upload_frames_yuv": [P, P, S, S, P, S, U64, P],
            "fvv_select_cameras": [C.POINTER(fvv_rig), I, C.POINTER(fvv_camera), I, C.POINTER(U64)],
            "fvv_depth_jbf": [P, S, P, S, P, S, I, I, C.POINTER(fvv_options), P],
            "fvv_latest_tick": [P, C.POINTER(U64)],
            "fvv_synthesize": [P, C.POINTER(fvv_camera), P, S, C.POINTER(fvv_aux), P],
            "fvv_synthesize_batch": [P, I, C.POINTER(fvv_camera), C.POINTER(U64), C.POINTER(P),
                                     C.POINTER(S), C.POINTER(fvv_aux), P],
            "fvv_view_params": [C.POINTER(fvv_rig), C.POINTER(fvv_options), C.POINTER(fvv_camera),
                                P, P, P],
            "fvv_synthesize_noalloc": [C.POINTER(fvv_rig), C.POINTER(fvv_options), C.POINTER(P),
                                       C.POINTER(S), C.POINTER(P), C.POINTER(S),
                                       C.POINTER(fvv_camera), P, S, P],
            "fvv_serve_default_cfg": [C.POINTER(fvv_serve_cfg)],
            "fvv_serve_start": [P, C.POINTER(fvv_serve_cfg)],
            "fvv_serve_submit": [P, C.c_uint32, C.POINTER(fvv_camera), P, S, C.POINTER(U64)],
            "fvv_serve_poll": [P, U64, C.c_int64],
            "fvv_serve_stats": [P, C.POINTER(fvv_serve_report), I],
            "fvv_serve_stop": [P],
            "fvv_unet_conv3x3": [P, I, I, I, I, P, P, I, I, P, P, P],
            "fvv_unet_wgrad3x3": [P, I, I, I, I, I, P, I, P, P, P],
            "fvv_selftest_bounded_wait": [I, C.c_uint32, P],
            "fvv_selftest_persistent_wait": [I, C.c_uint32, P],
            "fvv_unet_conv3x3_e4m3": [P, I, I, I, I, P, P, I, I, C.c_float, C.c_float, P, P],
            "fvv_unet_conv3x3_pool": [P, I, I, I, I, P, P, I, I, C.c_float, C.c_float, P, P, P, P],
            "fvv_depth_codec_default": [C.POINTER(fvv_depth_codec)],
            "fvv_set_depth_codec": [P, I, C.POINTER(fvv_depth_codec)],
            "fvv_depth_encode_yuv": [P, I, P, S, P, S, P, P, S, P],
            "fvv_depth_decode_yuv": [P, I, P, S, P, P, S, P, S, P],
            "fvv_depth_decode_yuv_frames": [P, I, P, S, P, S, S, P],
            "fvv_upload_frame_yuv": [P, I, P, S, P, S, P, P, S, U64, P],
            "fvv_refine_quantize": [P, C.POINTER(fvv_refine_batch), P, P],
            "fvv_refine_set_precision": [P, I],
            "fvv_refine_get_precision": [P, C.POINTER(I), P],
            "fvv_refine_default_cfg": [C.POINTER(fvv_unet_cfg)],
            "fvv_refine_init": [P, C.POINTER(fvv_unet_cfg)],
            "fvv_refine_param_count": [P, C.POINTER(U64)],
            "fvv_refine_get": [P, I, P],
            "fvv_refine_set": [P, I, P],
            "fvv_refine_forward": [P, C.POINTER(fvv_refine_batch), P, P, P],
            "fvv_refine_train_step": [P, C.POINTER(fvv_refine_batch), C.c_float, C.POINTER(C.c_float), P],
            "fvv_refine_save": [P, C.c_char_p],
            "fvv_refine_load": [P, C.c_char_p],
            "fvv_synthesize_refined": [P, C.POINTER(fvv_camera), P, S, P],
            "fvv_profile_enable": [P, I],
            "fvv_profile_read": [P, C.POINTER(fvv_kernel_stats), C.POINTER(I), I],
        }
        for name, args in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = C.c_char_p if name == "fvv_last_error" else C.c_int32
        _lib = lib
        return lib


def header_symbols() -> list:
    """Function names declared in include/fvv.h."""
    hdr = os.path.join(_build.INCLUDE, "fvv.h")
    text = open(hdr).read()
    return sorted(set(re.findall(r"^\s*(?:fvv_status|const char\*)\s+(fvv_\w+)\s*\(", text, re.M)))


def _check(code: int, func: str):
    if code != FVV_OK:
        msg = load().fvv_last_error()
        raise FvvError(code, func, msg.decode() if msg else "")


def ptr(x) -> Optional[int]:
    """Data pointer of an int / numpy array / torch tensor (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    raise TypeError("cannot take a pointer of %r" % type(x))


def stream_handle(stream) -> Optional[int]:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def camera(c) -> fvv_camera:
    """fvv_camera from any object with width, height, fx, fy, cx, cy, R, t."""
    out = fvv_camera()
    out.width, out.height = int(c.width), int(c.height)
    out.fx, out.fy, out.cx, out.cy = float(c.fx), float(c.fy), float(c.cx), float(c.cy)
    R = np.asarray(c.R, dtype=np.float64).reshape(9)
    t = np.asarray(c.t, dtype=np.float64).reshape(3)
    out.R[:] = [float(v) for v in R]
    out.t[:] = [float(v) for v in t]
    return out


def rig(cams: Sequence, look_at, depth_unit_m: float = 0.001) -> fvv_rig:
    arr = (fvv_camera * len(cams))(*[camera(c) for c in cams])
    r = fvv_rig()
    r.n_cams = len(cams)
    r.cams = C.cast(arr, C.POINTER(fvv_camera))
    r.look_at[:] = [float(v) for v in np.asarray(look_at, dtype=np.float64).reshape(3)]
    r.depth_unit_m = float(depth_unit_m)
    r._keep = arr
    return r


def fvv_default_options(**overrides) -> fvv_options:
    o = fvv_options()
    _check(load().fvv_default_options(C.byref(o)), "fvv_default_options")
    for k, v in overrides.items():
        if not hasattr(o, k):
            raise AttributeError(k)
        setattr(o, k, v)
    return o


def fvv_last_error() -> str:
    m = load().fvv_last_error()
    return m.decode() if m else ""


def fvv_create(rig_: fvv_rig, opt: Optional[fvv_options] = None) -> int:
    h = C.c_void_p()
    _check(load().fvv_create(C.byref(rig_), C.byref(opt) if opt is not None else None,
                             C.byref(h)), "fvv_create")
    return h.value


def fvv_destroy(ctx: int) -> None:
    _check(load().fvv_destroy(ctx), "fvv_destroy")


def fvv_upload_frame(ctx: int, cam: int, rgb, rgb_pitch: int, depth, depth_pitch: int,
                     tick: int, stream=None) -> None:
    _check(load().fvv_upload_frame(ctx, cam, ptr(rgb), rgb_pitch, ptr(depth), depth_pitch,
                                   tick, stream_handle(stream)), "fvv_upload_frame")


def fvv_depth_jbf(rgb, rgb_pitch: int, depth, depth_pitch: int, out, out_pitch: int, width: int, height: int,
                  opt: fvv_options, stream=None) -> None:
    """Joint bilateral depth pre-filter of one frame (device buffers)."""
    _check(load().fvv_depth_jbf(ptr(rgb), rgb_pitch, ptr(depth), depth_pitch, ptr(out), out_pitch, width, height,
                                C.byref(opt), stream_handle(stream)), "fvv_depth_jbf")


def fvv_upload_frames_subset(ctx: int, cam_mask: int, rgb, rgb_cam_stride: int, rgb_pitch: int, depth,
                             depth_cam_stride: int, depth_pitch: int, tick: int, stream=None) -> None:
    """The cameras of cam_mask for one tick, blocks packed in camera order."""
    _check(load().fvv_upload_frames_subset(ctx, cam_mask, ptr(rgb), rgb_cam_stride, rgb_pitch, ptr(depth),
                                           depth_cam_stride, depth_pitch, tick, stream_handle(stream)),
           "fvv_upload_frames_subset")


def fvv_upload_frames_yuv(ctx: int, rgb, rgb_cam_stride: int, rgb_pitch: int, yuv, yuv_cam_stride: int, tick: int,
                          stream=None) -> None:
    """Every camera of one tick with dense planar YUV420 depth frames."""
    _check(load().fvv_upload_frames_yuv(ctx, ptr(rgb), rgb_cam_stride, rgb_pitch, ptr(yuv), yuv_cam_stride, tick,
                                        stream_handle(stream)), "fvv_upload_frames_yuv")


def fvv_select_cameras(rig_: fvv_rig, views, n_tx: int) -> int:
    """Bit mask of the n_tx cameras nearest each view, OR-ed over the views."""
    vs = list(views)
    arr = (fvv_camera * len(vs))(*[v if isinstance(v, fvv_camera) else camera(v) for v in vs])
    m = C.c_uint64()
    _check(load().fvv_select_cameras(C.byref(rig_), len(vs), arr, n_tx, C.byref(m)), "fvv_select_cameras")
    return m.value


def fvv_set_bg_depth(ctx: int, cam: int, depth, pitch: int = 0) -> None:
    """Camera `cam`'s static background depth model (None removes it)."""
    _check(load().fvv_set_bg_depth(ctx, cam, ptr(depth) if depth is not None else None, pitch),
           "fvv_set_bg_depth")


def fvv_upload_frames(ctx: int, rgb, rgb_cam_stride: int, rgb_pitch: int, depth,
                      depth_cam_stride: int, depth_pitch: int, tick: int, stream=None) -> None:
    _check(load().fvv_upload_frames(ctx, ptr(rgb), rgb_cam_stride, rgb_pitch, ptr(depth),
                                    depth_cam_stride, depth_pitch, tick, stream_handle(stream)),
           "fvv_upload_frames")


def fvv_latest_tick(ctx: int) -> int:
    t = C.c_uint64()
    _check(load().fvv_latest_tick(ctx, C.byref(t)), "fvv_latest_tick")
    return t.value


def aux(depth=None, hole=None, top3=None, keys=None, keys_raw=None) -> fvv_aux:
    a = fvv_aux()
    a.depth, a.hole, a.top3, a.keys, a.keys_raw = (ptr(depth), ptr(hole), ptr(top3), ptr(keys),
                                                   ptr(keys_raw))
    return a


def fvv_synthesize(ctx: int, view, out_rgb, out_pitch: int, aux_: Optional[fvv_aux] = None,
                   stream=None) -> None:
    v = view if isinstance(view, fvv_camera) else camera(view)
    _check(load().fvv_synthesize(ctx, C.byref(v), ptr(out_rgb), out_pitch,
                                 C.byref(aux_) if aux_ is not None else None,
                                 stream_handle(stream)), "fvv_synthesize")


def fvv_synthesize_batch(ctx: int, views: Sequence, ticks: Optional[Sequence[int]], out_rgb: Sequence,
                         out_pitch: Sequence[int], aux_: Optional[Sequence[fvv_aux]] = None,
                         stream=None) -> None:
    n = len(views)
    va = (fvv_camera * n)(*[v if isinstance(v, fvv_camera) else camera(v) for v in views])
    ta = (C.c_uint64 * n)(*ticks) if ticks is not None else None
    oa = (C.c_void_p * n)(*[ptr(o) for o in out_rgb])
    pa = (C.c_size_t * n)(*out_pitch)
    aa = (fvv_aux * n)(*aux_) if aux_ is not None else None
    _check(load().fvv_synthesize_batch(ctx, n, va, ta, oa, pa, aa, stream_handle(stream)),
           "fvv_synthesize_batch")


def fvv_view_params(rig_: fvv_rig, opt: Optional[fvv_options], view):
    """Host-only composition: returns M (K,3,4), N (K,3,4), w (K,) as float32."""
    K = rig_.n_cams
    M = np.zeros((K, 3, 4), np.float32)
    N = np.zeros((K, 3, 4), np.float32)
    w = np.zeros(K, np.float32)
    v = view if isinstance(view, fvv_camera) else camera(view)
    _check(load().fvv_view_params(C.byref(rig_), C.byref(opt) if opt is not None else None,
                                  C.byref(v), M.ctypes.data, N.ctypes.data, w.ctypes.data),
           "fvv_view_params")
    return M, N, w


def fvv_profile_enable(ctx: int, on: bool = True) -> None:
    _check(load().fvv_profile_enable(ctx, 1 if on else 0), "fvv_profile_enable")


def fvv_profile_read(ctx: int, reset: bool = False) -> dict:
    """{kernel name: (launches, timed launches, total ms)}."""
    n = C.c_int32(8)
    arr = (fvv_kernel_stats * 8)()
    _check(load().fvv_profile_read(ctx, arr, C.byref(n), 1 if reset else 0), "fvv_profile_read")
    return {arr[i].name.decode(): (arr[i].launches, arr[i].timed, arr[i].total_ms)
            for i in range(min(n.value, 8))}


def fvv_synthesize_noalloc(rig_: fvv_rig, opt: Optional[fvv_options], depth: Sequence,
                           depth_pitch: Sequence[int], rgba: Sequence, rgba_pitch: Sequence[int],
                           view, out_rgb, out_pitch: int, stream=None) -> None:
    """Allocation-free synthesis of one view from device frames (RGBA8 + uint16)."""
    n = rig_.n_cams
    dp = (C.c_void_p * n)(*[ptr(d) for d in depth])
    ds = (C.c_size_t * n)(*depth_pitch)
    rp = (C.c_void_p * n)(*[ptr(r) for r in rgba])
    rs = (C.c_size_t * n)(*rgba_pitch)
    v = view if isinstance(view, fvv_camera) else camera(view)
    _check(load().fvv_synthesize_noalloc(C.byref(rig_), C.byref(opt) if opt is not None else None,
                                         dp, ds, rp, rs, C.byref(v), ptr(out_rgb), out_pitch,
                                         stream_handle(stream)), "fvv_synthesize_noalloc")


def fvv_serve_default_cfg(**overrides) -> fvv_serve_cfg:
    cfg = fvv_serve_cfg()
    _check(load().fvv_serve_default_cfg(C.byref(cfg)), "fvv_serve_default_cfg")
    for k, v in overrides.items():
        if not hasattr(cfg, k):
            raise AttributeError(k)
        setattr(cfg, k, v)
    return cfg


def fvv_serve_start(ctx: int, cfg: Optional[fvv_serve_cfg] = None) -> None:
    _check(load().fvv_serve_start(ctx, C.byref(cfg) if cfg is not None else None), "fvv_serve_start")


def fvv_serve_submit(ctx: int, viewer: int, view, out, pitch: int) -> int:
    v = view if isinstance(view, fvv_camera) else camera(view)
    t = C.c_uint64()
    _check(load().fvv_serve_submit(ctx, viewer, C.byref(v), ptr(out), pitch, C.byref(t)),
           "fvv_serve_submit")
    return t.value


def fvv_serve_poll(ctx: int, ticket: int, timeout_us: int = -1) -> None:
    _check(load().fvv_serve_poll(ctx, ticket, timeout_us), "fvv_serve_poll")


def fvv_serve_stats(ctx: int, reset: bool = False) -> dict:
    r = fvv_serve_report()
    _check(load().fvv_serve_stats(ctx, C.byref(r), 1 if reset else 0), "fvv_serve_stats")
    return {f: getattr(r, f) for f, _ in fvv_serve_report._fields_}


def fvv_serve_stop(ctx: int) -> None:
    _check(load().fvv_serve_stop(ctx), "fvv_serve_stop")


def fvv_unet_wgrad3x3(x, n: int, h: int, w: int, cin: int, xstride: int, dz, cout: int, dw, db,
                      stream=None) -> None:
    """Weight (and bias) gradients of a 3x3 convolution on the tensor cores."""
    _check(load().fvv_unet_wgrad3x3(ptr(x), n, h, w, cin, xstride, ptr(dz), cout, ptr(dw), ptr(db),
                                    stream_handle(stream)), "fvv_unet_wgrad3x3")


def fvv_unet_conv3x3(x, n: int, h: int, w: int, cin: int, wt, bias, cout: int, relu: bool, mask, y,
                     stream=None) -> None:
    _check(load().fvv_unet_conv3x3(ptr(x), n, h, w, cin, ptr(wt), ptr(bias), cout, 1 if relu else 0,
                                   ptr(mask), ptr(y), stream_handle(stream)), "fvv_unet_conv3x3")


def fvv_unet_conv3x3_e4m3(x, n: int, h: int, w: int, cin: int, wt, bias, cout: int, relu: bool,
                          acc_scale: float, out_inv_scale: float, y, stream=None) -> None:
    _check(load().fvv_unet_conv3x3_e4m3(ptr(x), n, h, w, cin, ptr(wt), ptr(bias), cout, 1 if relu else 0,
                                        acc_scale, out_inv_scale, ptr(y), stream_handle(stream)),
           "fvv_unet_conv3x3_e4m3")


def fvv_unet_conv3x3_pool(x, n: int, h: int, w: int, cin: int, wt, bias, cout: int, y, pool_y, pool_arg=None,
                          e4m3: bool = False, acc_scale: float = 1.0, out_inv_scale: float = 1.0,
                          stream=None) -> None:
    _check(load().fvv_unet_conv3x3_pool(ptr(x), n, h, w, cin, ptr(wt), ptr(bias), cout, 1 if e4m3 else 0,
                                        acc_scale, out_inv_scale, ptr(y), ptr(pool_y), ptr(pool_arg),
                                        stream_handle(stream)), "fvv_unet_conv3x3_pool")


class fvv_depth_codec(C.Structure):
    _fields_ = [("z_near", C.c_double), ("z_far", C.c_double), ("alpha", C.c_double), ("beta", C.c_double)]


def fvv_depth_codec_default(**overrides) -> fvv_depth_codec:
    k = fvv_depth_codec()
    _check(load().fvv_depth_codec_default(C.byref(k)), "fvv_depth_codec_default")
    for n, v in overrides.items():
        setattr(k, n, v)
    return k


def fvv_set_depth_codec(ctx: int, cam: int, codec: fvv_depth_codec) -> None:
    _check(load().fvv_set_depth_codec(ctx, cam, C.byref(codec)), "fvv_set_depth_codec")


def fvv_depth_encode_yuv(ctx: int, cam: int, depth, depth_pitch: int, y, y_pitch: int, u, v, uv_pitch: int,
                         stream=None) -> None:
    _check(load().fvv_depth_encode_yuv(ctx, cam, ptr(depth), depth_pitch, ptr(y), y_pitch, ptr(u), ptr(v),
                                       uv_pitch, stream_handle(stream)), "fvv_depth_encode_yuv")


def fvv_depth_decode_yuv(ctx: int, cam: int, y, y_pitch: int, u, v, uv_pitch: int, depth, depth_pitch: int,
                         stream=None) -> None:
    _check(load().fvv_depth_decode_yuv(ctx, cam, ptr(y), y_pitch, ptr(u), ptr(v), uv_pitch, ptr(depth),
                                       depth_pitch, stream_handle(stream)), "fvv_depth_decode_yuv")


def fvv_depth_decode_yuv_frames(ctx: int, n_cams: int, yuv, yuv_cam_stride: int, depth, depth_cam_stride: int,
                                depth_pitch: int, stream=None) -> None:
    _check(load().fvv_depth_decode_yuv_frames(ctx, n_cams, ptr(yuv), yuv_cam_stride, ptr(depth), depth_cam_stride,
                                              depth_pitch, stream_handle(stream)), "fvv_depth_decode_yuv_frames")


def fvv_upload_frame_yuv(ctx: int, cam: int, rgb, rgb_pitch: int, y, y_pitch: int, u, v, uv_pitch: int,
                         tick: int, stream=None) -> None:
    _check(load().fvv_upload_frame_yuv(ctx, cam, ptr(rgb), rgb_pitch, ptr(y), y_pitch, ptr(u), ptr(v), uv_pitch,
                                       tick, stream_handle(stream)), "fvv_upload_frame_yuv")


FVV_PREC_BF16 = 0
FVV_PREC_E4M3 = 1


def fvv_refine_quantize(ctx: int, calib=None, act_scales=None, stream=None) -> None:
    """E4M3 inference from now on: scales from a bf16 pass over `calib`
    (a refine_batch), or the ten given activation scales."""
    sc = None
    if act_scales is not None:
        sc = np.ascontiguousarray(act_scales, np.float32)
        assert sc.size == 10
    _check(load().fvv_refine_quantize(ctx, C.byref(calib) if calib is not None else None,
                                      sc.ctypes.data if sc is not None else None, stream_handle(stream)),
           "fvv_refine_quantize")


def fvv_refine_set_precision(ctx: int, precision: int) -> None:
    _check(load().fvv_refine_set_precision(ctx, precision), "fvv_refine_set_precision")


def fvv_refine_get_precision(ctx: int):
    p = C.c_int32()
    sc = np.zeros(10, np.float32)
    _check(load().fvv_refine_get_precision(ctx, C.byref(p), sc.ctypes.data), "fvv_refine_get_precision")
    return p.value, sc


def fvv_selftest_bounded_wait(arrive: bool, limit_us: int, stream=None) -> int:
    """Returns the raw status (FVV_OK or FVV_ERR_TIMEOUT are both expected
    outcomes); other failures raise."""
    st = load().fvv_selftest_bounded_wait(1 if arrive else 0, limit_us, stream_handle(stream))
    if st not in (FVV_OK, FVV_ERR_TIMEOUT):
        _check(st, "fvv_selftest_bounded_wait")
    return st


def fvv_selftest_persistent_wait(barrier: bool, limit_us: int, stream=None) -> int:
    """Returns the raw status (FVV_ERR_TIMEOUT is the expected outcome);
    other failures raise."""
    st = load().fvv_selftest_persistent_wait(1 if barrier else 0, limit_us, stream_handle(stream))
    if st != FVV_ERR_TIMEOUT:
        _check(st, "fvv_selftest_persistent_wait")
    return st


def fvv_refine_default_cfg(**overrides) -> fvv_unet_cfg:
    cfg = fvv_unet_cfg()
    _check(load().fvv_refine_default_cfg(C.byref(cfg)), "fvv_refine_default_cfg")
    for k, v in overrides.items():
        if k == "widths":
            cfg.widths[:] = list(v)
        else:
            setattr(cfg, k, v)
    return cfg


def fvv_refine_init(ctx: int, cfg: Optional[fvv_unet_cfg] = None) -> None:
    _check(load().fvv_refine_init(ctx, C.byref(cfg) if cfg is not None else None), "fvv_refine_init")


def fvv_refine_param_count(ctx: int) -> int:
    n = C.c_uint64()
    _check(load().fvv_refine_param_count(ctx, C.byref(n)), "fvv_refine_param_count")
    return n.value


def fvv_refine_get(ctx: int, which: int = FVV_REFINE_PARAMS) -> np.ndarray:
    out = np.zeros(fvv_refine_param_count(ctx), np.float32)
    _check(load().fvv_refine_get(ctx, which, out.ctypes.data), "fvv_refine_get")
    return out


def fvv_refine_set(ctx: int, which: int, values) -> None:
    v = np.ascontiguousarray(values, dtype=np.float32)
    _check(load().fvv_refine_set(ctx, which, v.ctypes.data), "fvv_refine_set")


def refine_batch(n, height, width, rgb, depth, hole, top3, target=None) -> fvv_refine_batch:
    b = fvv_refine_batch()
    b.n, b.height, b.width = n, height, width
    b.rgb, b.depth, b.hole, b.top3, b.target = ptr(rgb), ptr(depth), ptr(hole), ptr(top3), ptr(target)
    return b


def fvv_refine_forward(ctx: int, batch: fvv_refine_batch, out_rgb=None, out_f32=None, stream=None) -> None:
    _check(load().fvv_refine_forward(ctx, C.byref(batch), ptr(out_rgb), ptr(out_f32),
                                     stream_handle(stream)), "fvv_refine_forward")


def fvv_refine_train_step(ctx: int, batch: fvv_refine_batch, lr: float, stream=None) -> float:
    loss = C.c_float()
    _check(load().fvv_refine_train_step(ctx, C.byref(batch), lr, C.byref(loss), stream_handle(stream)),
           "fvv_refine_train_step")
    return loss.value


def fvv_refine_save(ctx: int, path: str) -> None:
    _check(load().fvv_refine_save(ctx, path.encode()), "fvv_refine_save")


def fvv_refine_load(ctx: int, path: str) -> None:
    _check(load().fvv_refine_load(ctx, path.encode()), "fvv_refine_load")


def fvv_synthesize_refined(ctx: int, view, out_rgb, out_pitch: int, stream=None) -> None:
    v = view if isinstance(view, fvv_camera) else camera(view)
    _check(load().fvv_synthesize_refined(ctx, C.byref(v), ptr(out_rgb), out_pitch, stream_handle(stream)),
           "fvv_synthesize_refined")
