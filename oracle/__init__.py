"""CPU oracle of FVV Live's view synthesis (Sec. VI), plain C behind ctypes.

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by
the benchmark's CPU-baseline leg; never by the library.  It shares no code
with the CUDA path.  ``build()`` compiles ``fvv_oracle.c`` with gcc
(FMA contraction off, no fast-math) into ``oracle/_build/``.

Every step is pinned by the CPU tests in ``tests/test_oracle_*.py`` against
facts the method and the geometry fix (identity pose, f B / Z shift,
brute-force z-buffer, analytic ray-cast, hand-built filter/blend/fill cases).
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fvv_oracle.c")
_HDR = os.path.join(_HERE, "fvv_oracle.h")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

KEY_EMPTY = np.uint64(0xFFFFFFFFFFFFFFFF)
SRC_BITS = 26
DEPTH_BG = 65535      # depth code signalling a background pixel (Sec. V-A, 12-bit code 0)

CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
          "-shared", "-Wall", "-Wextra"]


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc); returns its path."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < newest:
        tmp = _OUT + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", *CFLAGS, _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _OUT)
    return _OUT


class Camera(C.Structure):
    _fields_ = [("width", C.c_int), ("height", C.c_int),
                ("fx", C.c_double), ("fy", C.c_double), ("cx", C.c_double), ("cy", C.c_double),
                ("R", C.c_double * 9), ("t", C.c_double * 3)]


class Options(C.Structure):
    _fields_ = [("n_ref", C.c_int), ("crack_filter", C.c_int), ("hole_fill", C.c_int),
                ("tau_crack", C.c_float), ("tau_vis", C.c_float), ("z_min", C.c_float),
                ("d_lo", C.c_uint32), ("d_hi", C.c_uint32), ("pixel_weights", C.c_int)]


class XForm(C.Structure):
    _fields_ = [("M", C.c_float * 12), ("N", C.c_float * 12), ("w", C.c_float),
                ("cv", C.c_float * 3), ("vk", C.c_float * 4)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P = C.c_void_p
            lib.oracle_default_options.argtypes = [C.POINTER(Options)]
            lib.oracle_compose.argtypes = [C.c_int, C.POINTER(Camera), C.POINTER(Camera), P,
                                           C.c_double, C.c_int, C.POINTER(XForm)]
            lib.oracle_warp_splat.argtypes = [C.c_int, C.POINTER(Camera), P, P, C.POINTER(XForm),
                                              C.c_int, C.c_int, C.POINTER(Options), P]
            lib.oracle_crack_filter.argtypes = [P, C.c_int, C.c_int, C.c_float, P]
            lib.oracle_fetch_blend.argtypes = [C.c_int, C.POINTER(Camera), P, P, P, P,
                                               C.POINTER(XForm), P, C.c_int, C.c_int,
                                               C.POINTER(Options), P, P, P, P, P]
            lib.oracle_hole_fill.argtypes = [C.c_int, C.c_int, P, P, P]
            lib.oracle_synthesize.argtypes = [C.c_int, C.POINTER(Camera), P, P, P, P, P,
                                              C.c_double, C.POINTER(Camera), C.POINTER(Options),
                                              P, P, P, P, P, P]
            lib.oracle_synthesize.restype = C.c_int
            _lib = lib
    return _lib


def _cam(c) -> Camera:
    out = Camera()
    out.width, out.height = int(c.width), int(c.height)
    out.fx, out.fy, out.cx, out.cy = float(c.fx), float(c.fy), float(c.cx), float(c.cy)
    R = np.ascontiguousarray(np.asarray(c.R, dtype=np.float64).reshape(9))
    t = np.ascontiguousarray(np.asarray(c.t, dtype=np.float64).reshape(3))
    for i in range(9):
        out.R[i] = R[i]
    for i in range(3):
        out.t[i] = t[i]
    return out


def _cams(cams) -> C.Array:
    arr = (Camera * len(cams))()
    for i, c in enumerate(cams):
        arr[i] = _cam(c)
    return arr


def options(**kw) -> Options:
    o = Options()
    _load().oracle_default_options(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _frames(rgb, depth, n):
    """Per-camera contiguous arrays plus pointer and pitch tables."""
    rl = [np.ascontiguousarray(rgb[k], dtype=np.uint8) for k in range(n)]
    dl = [np.ascontiguousarray(depth[k], dtype=np.uint16) for k in range(n)]
    rp = (C.c_void_p * n)(*[_ptr(a) for a in rl])
    dp = (C.c_void_p * n)(*[_ptr(a) for a in dl])
    rpitch = (C.c_size_t * n)(*[a.shape[1] * 3 for a in rl])
    dpitch = (C.c_size_t * n)(*[a.shape[1] * 2 for a in dl])
    return rl, dl, rp, dp, rpitch, dpitch


def compose(cams, view, look_at, depth_unit_m: float = 0.001, n_ref: int = 0):
    """FP64 composition rounded to FP32: returns M (K,3,4), N (K,3,4), w (K,)."""
    lib = _load()
    n = len(cams)
    xf = (XForm * n)()
    la = np.ascontiguousarray(np.asarray(look_at, dtype=np.float64).reshape(3))
    vc = _cam(view)
    lib.oracle_compose(n, _cams(cams), C.byref(vc), _ptr(la), depth_unit_m, n_ref, xf)
    M = np.array([list(x.M) for x in xf], dtype=np.float32).reshape(n, 3, 4)
    N = np.array([list(x.N) for x in xf], dtype=np.float32).reshape(n, 3, 4)
    w = np.array([x.w for x in xf], dtype=np.float32)
    return M, N, w


def compose_pixel(cams, view, look_at, depth_unit_m: float = 0.001):
    """The per-pixel weight inputs of the composition (R9): each camera's
    centre in the view's frame (K, 3) and the view's (cx, cy, 1/fx, 1/fy),
    FP32."""
    lib = _load()
    n = len(cams)
    xf = (XForm * n)()
    la = np.ascontiguousarray(np.asarray(look_at, dtype=np.float64).reshape(3))
    vc = _cam(view)
    lib.oracle_compose(n, _cams(cams), C.byref(vc), _ptr(la), depth_unit_m, 0, xf)
    cv = np.array([list(x.cv) for x in xf], dtype=np.float32)
    return cv, np.array(list(xf[0].vk), dtype=np.float32)


def _xf(M, N, w, cv=None, vk=None):
    n = len(w)
    xf = (XForm * n)()
    for k in range(n):
        for i in range(12):
            xf[k].M[i] = float(np.float32(M[k].reshape(12)[i]))
            xf[k].N[i] = float(np.float32(N[k].reshape(12)[i]))
        xf[k].w = float(np.float32(w[k]))
        if cv is not None:
            for i in range(3):
                xf[k].cv[i] = float(cv[k][i])
            for i in range(4):
                xf[k].vk[i] = float(vk[i])
    return xf


def warp_splat(cams, depth, M, w, Wv: int, Hv: int, opts: Optional[Options] = None,
               N=None) -> np.ndarray:
    """Steps a + b: raw z-buffer keys (Hv, Wv) uint64."""
    lib = _load()
    n = len(cams)
    opts = opts or options()
    dl = [np.ascontiguousarray(depth[k], dtype=np.uint16) for k in range(n)]
    dp = (C.c_void_p * n)(*[_ptr(a) for a in dl])
    dpitch = (C.c_size_t * n)(*[a.shape[1] * 2 for a in dl])
    keys = np.empty((Hv, Wv), dtype=np.uint64)
    N = M if N is None else N
    lib.oracle_warp_splat(n, _cams(cams), dp, dpitch, _xf(M, N, w), Wv, Hv,
                          C.byref(opts), _ptr(keys))
    return keys


def crack_filter(keys: np.ndarray, tau: float = 0.05) -> np.ndarray:
    """Step c: one out-of-place pass of the 3x3 crack/outlier rule."""
    lib = _load()
    k = np.ascontiguousarray(keys, dtype=np.uint64)
    out = np.empty_like(k)
    lib.oracle_crack_filter(_ptr(k), k.shape[1], k.shape[0], tau, _ptr(out))
    return out


def fetch_blend(cams, rgb, depth, M, N, w, keys, opts: Optional[Options] = None, cv=None, vk=None):
    """Step d: returns dict(rgb, depth, hole, top3, nvis) before hole fill
    (with opts.pixel_weights, cv and vk from compose_pixel)."""
    lib = _load()
    n = len(cams)
    opts = opts or options()
    rl, dl, rp, dp, rpitch, dpitch = _frames(rgb, depth, n)
    k = np.ascontiguousarray(keys, dtype=np.uint64)
    Hv, Wv = k.shape
    out = np.zeros((Hv, Wv, 3), np.uint8)
    dep = np.zeros((Hv, Wv), np.float32)
    hole = np.zeros((Hv, Wv), np.uint8)
    top3 = np.zeros((Hv, Wv, 3), np.float32)
    nvis = np.zeros((Hv, Wv), np.uint8)
    lib.oracle_fetch_blend(n, _cams(cams), rp, rpitch, dp, dpitch, _xf(M, N, w, cv, vk), _ptr(k),
                           Wv, Hv, C.byref(opts), _ptr(out), _ptr(dep), _ptr(hole),
                           _ptr(top3), _ptr(nvis))
    return {"rgb": out, "depth": dep, "hole": hole, "top3": top3, "nvis": nvis}


def hole_fill(hole, rgb, depth):
    """Step e on copies of ``rgb`` (H, W, 3) and ``depth`` (H, W)."""
    lib = _load()
    h = np.ascontiguousarray(hole, dtype=np.uint8)
    r = np.array(rgb, dtype=np.uint8, order="C", copy=True)
    d = np.array(depth, dtype=np.float32, order="C", copy=True)
    lib.oracle_hole_fill(h.shape[1], h.shape[0], _ptr(h), _ptr(r), _ptr(d))
    return r, d


def synthesize(cams: Sequence, rgb, depth, view, look_at, opts: Optional[Options] = None,
               depth_unit_m: float = 0.001, **kw) -> dict:
    """All steps a-e for one virtual view.

    ``rgb[k]`` is (H_k, W_k, 3) uint8, ``depth[k]`` (H_k, W_k) uint16 in depth
    units.  Returns dict(rgb, depth, hole, top3, keys_raw, keys).
    """
    lib = _load()
    n = len(cams)
    if opts is None:
        opts = options(**kw)
    rl, dl, rp, dp, rpitch, dpitch = _frames(rgb, depth, n)
    Hv, Wv = int(view.height), int(view.width)
    out = np.zeros((Hv, Wv, 3), np.uint8)
    dep = np.zeros((Hv, Wv), np.float32)
    hole = np.zeros((Hv, Wv), np.uint8)
    top3 = np.zeros((Hv, Wv, 3), np.float32)
    kr = np.empty((Hv, Wv), np.uint64)
    kf = np.empty((Hv, Wv), np.uint64)
    la = np.ascontiguousarray(np.asarray(look_at, dtype=np.float64).reshape(3))
    vc = _cam(view)
    rc = lib.oracle_synthesize(n, _cams(cams), rp, rpitch, dp, dpitch, _ptr(la), depth_unit_m,
                               C.byref(vc), C.byref(opts), _ptr(out), _ptr(dep), _ptr(hole),
                               _ptr(top3), _ptr(kr), _ptr(kf))
    if rc != 0:
        raise ValueError("oracle_synthesize: invalid arguments")
    return {"rgb": out, "depth": dep, "hole": hole, "top3": top3, "keys_raw": kr, "keys": kf}


def select_cameras(cams: Sequence, views: Sequence, look_at, n_tx: int) -> int:
    """Adaptive view transmission (Sec. V-C): the n_tx cameras closest to
    each virtual viewpoint, OR-ed over the views, as a bit mask.  Closeness
    is the angle the blend weights use, between the directions from the
    rig's look-at point O to the two camera centres, atan2(|a x b|, a . b)
    in FP64; ties go to the lower camera index."""
    O = np.asarray(look_at, dtype=np.float64).reshape(3)
    centres = [-(np.asarray(c.R, np.float64).T @ np.asarray(c.t, np.float64)) for c in cams]
    mask = 0
    for v in views:
        a = -(np.asarray(v.R, np.float64).T @ np.asarray(v.t, np.float64)) - O
        th = []
        for C in centres:
            b = C - O
            th.append(math.atan2(float(np.linalg.norm(np.cross(a, b))), float(a @ b)))
        order = sorted(range(len(cams)), key=lambda k: (th[k], k))
        for k in order[:n_tx]:
            mask |= 1 << k
    return mask


def synthesize_layered(cams: Sequence, rgb, depth, bg, view, look_at, opts: Optional[Options] = None,
                       depth_unit_m: float = 0.001, **kw) -> dict:
    """Layered FG/BG synthesis of one virtual view (Sec. VI, the per-camera
    FG and BG layers and their mixing and stacking), composed from steps a-e.

    ``depth[k]`` holds camera k's live codes, ``DEPTH_BG`` where the pixel
    is background; ``bg[k]`` its static background model (depth codes, 0 =
    none; ``bg`` or ``bg[k]`` may be None).  Readings taken here:

    * FG layer: every camera's live codes.  A BG-signalled pixel is no FG
      point because ``d_hi`` <= 65534 keeps ``DEPTH_BG`` out of the accepted
      codes; a pixel without depth (0) is in neither layer.
    * BG layer: camera k's model depth where camera k signals BG, 0 (no
      point) elsewhere -- where camera k sees a foreground object it holds no
      background colour.  The colour is always the live frame's.
    * Each layer goes through steps a-d on its own (z-buffer, crack filter,
      blend whose visibility test reads that layer's depth maps), with the
      weights of the one composition of the view.
    * Stacking: the FG layer where its filtered key is present, else the BG
      layer, else a hole; step e runs on the stacked image.

    Returns dict(rgb, depth, hole, top3, keys (key of the layer shown),
    keys_raw (the FG layer before the filter), keys_raw_bg, layer (0 FG,
    1 BG, -1 hole))."""
    n = len(cams)
    if opts is None:
        opts = options(**kw)
    if opts.d_hi >= DEPTH_BG:
        raise ValueError("layered synthesis needs d_hi <= 65534")
    Hv, Wv = int(view.height), int(view.width)
    M, N, w = compose(cams, view, look_at, depth_unit_m, opts.n_ref)
    cv, vk = compose_pixel(cams, view, look_at, depth_unit_m)
    live = [np.ascontiguousarray(depth[k], dtype=np.uint16) for k in range(n)]
    model = []
    for k in range(n):
        m = None if bg is None else bg[k]
        m = np.zeros_like(live[k]) if m is None else np.asarray(m, dtype=np.uint16)
        model.append(np.where(live[k] == DEPTH_BG, m, 0).astype(np.uint16))
    layers = []
    for dmaps in (live, model):
        raw = warp_splat(cams, dmaps, M, w, Wv, Hv, opts, N)
        filt = crack_filter(raw, opts.tau_crack) if opts.crack_filter else raw.copy()
        layers.append((raw, filt, fetch_blend(cams, rgb, dmaps, M, N, w, filt, opts, cv, vk)))
    (rf, kf, bf), (rb, kb, bb) = layers
    on_fg = kf != KEY_EMPTY
    on_bg = ~on_fg & (kb != KEY_EMPTY)
    pick = lambda a, b, fill: np.where(on_fg[..., None] if a.ndim == 3 else on_fg, a,
                                       np.where(on_bg[..., None] if b.ndim == 3 else on_bg, b, fill))
    out = pick(bf["rgb"], bb["rgb"], 0).astype(np.uint8)
    dep = pick(bf["depth"], bb["depth"], 0.0).astype(np.float32)
    top3 = pick(bf["top3"], bb["top3"], 0.0).astype(np.float32)
    hole = (~on_fg & ~on_bg).astype(np.uint8)
    if opts.hole_fill:
        out, dep = hole_fill(hole, out, dep)
    keys = np.where(on_fg, kf, kb)
    layer = np.where(on_fg, 0, np.where(on_bg, 1, -1)).astype(np.int8)
    return {"rgb": out, "depth": dep, "hole": hole, "top3": top3, "keys": keys, "keys_raw": rf,
            "keys_raw_bg": rb, "layer": layer}


def key_fields(keys: np.ndarray):
    """Split keys into (depth f32, camera, source index); empty -> (inf, -1, -1)."""
    k = np.asarray(keys, dtype=np.uint64)
    empty = k == KEY_EMPTY
    z = (k >> np.uint64(32)).astype(np.uint32).view(np.float32).copy()
    cam = ((k >> np.uint64(SRC_BITS)) & np.uint64(63)).astype(np.int64)
    src = (k & np.uint64((1 << SRC_BITS) - 1)).astype(np.int64)
    z[empty] = np.inf
    cam[empty] = -1
    src[empty] = -1
    return z, cam, src
