"""CPU tests of the boundary: libfvv.so builds and loads without a GPU, exports
every function include/fvv.h declares, validates arguments on the host, and
composes the per-view maps and weights bit-for-bit like the oracle."""
import ctypes

import numpy as np
import pytest

import synthetic as S
from fvv_helpers import lib


@pytest.fixture(scope="module")
def F():
    return lib()


def test_exports_every_declared_symbol(F):
    names = F.header_symbols()
    assert len(names) >= 10
    so = ctypes.CDLL(F.lib_path())
    for n in names:
        assert hasattr(so, n), "missing export " + n


def test_default_options(F):
    o = F.fvv_default_options()
    assert (o.n_ref, o.crack_filter, o.hole_fill) == (0, 1, 1)
    assert o.tau_crack == pytest.approx(0.05) and o.tau_vis == pytest.approx(0.03)
    assert (o.d_lo, o.d_hi, o.frame_slots, o.layered) == (1, 65534, 2, 0)


def _rigs():
    out = []
    w1 = S.rig_parallel(2, 320, 240, 300.0, 0.1)
    out.append((w1, S.rig_parallel(1, 320, 240, 300.0, 0.1)[0], [0, 0, 2.0]))
    cams = S.rig_arc(9, 90.0, 1.5, 1280, 720, 1000.0)
    for i in (0, 37, 150, 299):
        out.append((cams, S.trajectory_arc(300, 22.5, 1.5, 1280, 720, 1000.0)[i], [0, 0, 0]))
    out.append((cams, cams[3].copy(), [0, 0, 0]))
    # on camera 3's centre, turned 5 degrees about the vertical axis (not on it)
    a = np.radians(5.0)
    turn = np.array([[np.cos(a), 0.0, -np.sin(a)], [0.0, 1.0, 0.0], [np.sin(a), 0.0, np.cos(a)]])
    rot = cams[3].copy()
    rot.R, rot.t = turn @ cams[3].R, turn @ cams[3].t
    out.append((cams, rot, [0, 0, 0]))
    rng = np.random.default_rng(4)
    cams18 = S.rig_arc(18, 180.0, 2.0, 1920, 1080, 1500.0)
    for _ in range(3):
        out.append((cams18, S.arc_view(rng.uniform(-80, 80), rng.uniform(1.5, 2.5), 1920, 1080,
                                       rng.uniform(1200, 1800)), [0, 0, 0]))
    # non-square pixels (sources fy = 1.2 fx, the view fy = 0.9 fx), and the
    # rig moved off the origin with its look-at point
    sq = S.rig_arc(5, 60.0, 1.5, 640, 360, 500.0)
    for c in sq:
        c.fy = 1.2 * c.fx
    v = S.arc_view(7.0, 1.6, 640, 360, 520.0)
    v.fy = 0.9 * v.fx
    out.append((sq, v, [0, 0, 0]))
    off = np.array([1.0, -2.0, 3.0])
    mv = []
    for c in sq + [v]:
        m = c.copy()
        m.t = c.t - c.R @ off
        mv.append(m)
    out.append((mv[:-1], mv[-1], list(off)))
    return out


@pytest.mark.parametrize("n_ref", [0, 1, 3])
def test_view_params_match_oracle_bitwise(F, oracle_mod, n_ref):
    """The library's host-side FP64 composition rounds to the same FP32 maps
    and weights as the oracle's (independently written) composition."""
    for cams, view, O in _rigs():
        nr = min(n_ref, len(cams))
        M, N, w = F.fvv_view_params(F.rig(cams, O), F.fvv_default_options(n_ref=nr), view)
        Mo, No, wo = oracle_mod.compose(cams, view, O, n_ref=nr)
        assert np.array_equal(M.view(np.uint32), Mo.view(np.uint32))
        assert np.array_equal(N.view(np.uint32), No.view(np.uint32))
        assert np.array_equal(w.view(np.uint32), wo.view(np.uint32))


def _code(F, fn, *args):
    try:
        fn(*args)
    except F.FvvError as e:
        assert F.fvv_last_error() != ""
        return e.code
    return 0


def test_invalid_arguments_rejected_on_host(F):
    cams = S.rig_parallel(2, 32, 24, 30.0, 0.1)
    good = F.rig(cams, [0, 0, 1])
    # no cameras
    bad = F.rig(cams, [0, 0, 1])
    bad.n_cams = 0
    assert _code(F, F.fvv_create, bad) == F.FVV_ERR_INVALID_ARG
    bad.n_cams = 65
    assert _code(F, F.fvv_create, bad) == F.FVV_ERR_INVALID_ARG
    # bad depth unit
    bad = F.rig(cams, [0, 0, 1], depth_unit_m=0.0)
    assert _code(F, F.fvv_create, bad) == F.FVV_ERR_INVALID_ARG
    # source image too large for the 26-bit pixel field
    big = [c.copy() for c in cams]
    big[0].width, big[0].height = 8193, 8192
    assert _code(F, F.fvv_create, F.rig(big, [0, 0, 1])) == F.FVV_ERR_INVALID_ARG
    # non-finite pose
    nanc = [c.copy() for c in cams]
    nanc[1].t = np.array([np.nan, 0, 0])
    assert _code(F, F.fvv_view_params, F.rig(nanc, [0, 0, 1]), None, cams[0]) == F.FVV_ERR_INVALID_ARG
    # options
    for kw in ({"n_ref": 3}, {"tau_vis": -1.0}, {"d_lo": 0}, {"d_lo": 9, "d_hi": 8},
               {"d_hi": 65535}, {"layered": 2}, {"frame_slots": 0}, {"max_batch": 0}):
        assert _code(F, F.fvv_create, good, F.fvv_default_options(**kw)) == F.FVV_ERR_INVALID_ARG
    # bad view
    v = cams[0].copy()
    v.fx = 0.0
    assert _code(F, F.fvv_view_params, good, None, v) == F.FVV_ERR_INVALID_ARG
    # NULL context
    assert _code(F, F.fvv_destroy, None) == 0
    assert _code(F, F.fvv_latest_tick, None) == F.FVV_ERR_INVALID_ARG


def test_selftest_limit_checked_on_host(F):
    so = F.load()
    for lim in (0, 2000001):
        assert so.fvv_selftest_bounded_wait(0, lim, None) == F.FVV_ERR_INVALID_ARG


# Entry points that forward to another entry point (which holds the scope).
_FORWARDERS = {"fvv_synthesize": "fvv_synthesize_batch", "fvv_upload_frames": "fvv_upload_frames_subset"}


def test_context_entry_points_select_the_context_device():
    """Every C-ABI call on a context that touches the GPU makes the context's
    device current for the call (a DeviceScope, which also gives the
    caller's device back), so its launches, allocations and the check that
    caller buffers are this device's memory never follow whatever device
    the calling thread had current.  A static check over the sources: each
    such function's body holds a DeviceScope before its first CUDA call."""
    import os
    import re
    csrc = os.path.join(os.path.dirname(__file__), "..", "paper_2007_00558_gb300", "csrc")
    found = {}
    for fn in sorted(os.listdir(csrc)):
        if not fn.endswith(".cu"):
            continue
        src = open(os.path.join(csrc, fn)).read()
        for m in re.finditer(r"\nfvv_status (fvv_\w+)\(fvv_ctx\* c[,)]", src):
            name = m.group(1)
            start = src.index("{", m.end())
            depth, i = 0, start
            while True:
                if src[i] == "{":
                    depth += 1
                elif src[i] == "}":
                    depth -= 1
                    if depth == 0:
                        break
                i += 1
            found[name] = src[start:i]
    assert len(found) >= 30, sorted(found)
    missing = []
    for name, body in found.items():
        if name in _FORWARDERS:
            assert _FORWARDERS[name] + "(" in body and "cuda" not in body, name
            continue
        scope = body.find("DeviceScope")
        calls = [body.find(t) for t in ("cuda", "run_batch", "upload_", "launch_", "dev_alloc", "serve_shutdown",
                                        "refine_", "ensure_")]
        calls = [c for c in calls if c >= 0]
        if calls and (scope < 0 or min(calls) < scope):
            missing.append(name)
    assert not missing, "entry points without a device scope before their first CUDA call: %s" % missing
