"""The allocation-free entry point, fvv_synthesize_noalloc.

It serves callers that must not call cudaMalloc (a process whose device
memory belongs to another allocator, or a real-time render thread on which an
allocation would synchronise the device).  Its scratch is a fixed file-scope
device array.  These tests call it through the C ABI, two calls in a row on
the shared scratch, and check its colour byte for byte against both the
context-based fvv_synthesize (the same kernels) and the CPU oracle, for the
default options, per-pixel weights, the filter and fill switched off, padded
frame pitches and a caller's stream; a warmed-up call must leave the device's
free memory unchanged.  The file is collected last and passes both alone in a
fresh process and after the other tests.
"""
import numpy as np
import pytest

import synthetic as S
from fvv_helpers import lib

pytestmark = pytest.mark.gpu

VIEWS = (37, 150)


def _device_frames(wl, pad=0):
    """Frames in the library's device layout (uint16 depth, RGBA8 words), each
    row padded by ``pad`` elements; returns per-camera tensors and pitches."""
    import torch
    K = len(wl["cams"])
    H, W = wl["cams"][0].height, wl["cams"][0].width
    r = torch.from_numpy(np.ascontiguousarray(wl["rgb"])).cuda().to(torch.int32)
    words = r[..., 0] | (r[..., 1] << 8) | (r[..., 2] << 16)
    rgba = torch.zeros((K, H, W + pad), dtype=torch.int32, device="cuda")
    rgba[:, :, :W] = words
    depth = torch.zeros((K, H, W + pad), dtype=torch.int16, device="cuda")
    depth[:, :, :W] = torch.from_numpy(np.ascontiguousarray(wl["depth"]).view(np.int16)).cuda()
    return ([depth[k] for k in range(K)], [(W + pad) * 2] * K,
            [rgba[k] for k in range(K)], [(W + pad) * 4] * K)


@pytest.fixture(scope="module")
def arc():
    return S.workload("plain_9cam_1280x720")


def _context_views(F, wl, opts):
    """The same views through fvv_create / fvv_synthesize (device outputs)."""
    import torch
    cams = wl["cams"]
    K, H, W = len(cams), cams[0].height, cams[0].width
    ctx = F.fvv_create(F.rig(cams, wl["look_at"]), opts)
    refs = []
    try:
        for k in range(K):
            F.fvv_upload_frame(ctx, k, np.ascontiguousarray(wl["rgb"][k]), W * 3,
                               np.ascontiguousarray(wl["depth"][k]), W * 2, 0)
        for i in VIEWS:
            ref = torch.zeros((H, W * 3), dtype=torch.uint8, device="cuda")
            F.fvv_synthesize(ctx, wl["views"][i], ref, W * 3)
            refs.append(ref)
        torch.cuda.synchronize()
    finally:
        F.fvv_destroy(ctx)
    return [r.cpu().numpy().reshape(H, W, 3) for r in refs]


CASES = {
    "defaults": (dict(), 0, False),
    "pixel_weights": (dict(pixel_weights=1), 0, False),
    "no_filter_no_fill": (dict(crack_filter=0, hole_fill=0), 0, False),
    "padded_pitch": (dict(), 64, False),
    "caller_stream": (dict(), 0, True),
}


@pytest.mark.parametrize("case", list(CASES))
def test_noalloc_equals_synthesize_and_oracle_two_calls_in_a_row(arc, oracle_mod, case):
    import torch
    F = lib()
    wl = arc
    cams = wl["cams"]
    H, W = cams[0].height, cams[0].width
    over, pad, own_stream = CASES[case]
    opts = F.fvv_default_options(**over)
    rig = F.rig(cams, wl["look_at"])
    dp, dps, rp, rps = _device_frames(wl, pad)
    refs = _context_views(F, wl, opts)
    stream = torch.cuda.Stream() if own_stream else None
    outs = []
    for i in VIEWS:                            # two calls in a row, shared scratch
        out = torch.full((H, W * 3), 7, dtype=torch.uint8, device="cuda")
        F.fvv_synthesize_noalloc(rig, opts, dp, dps, rp, rps, wl["views"][i], out, W * 3, stream)
        outs.append(out)
    torch.cuda.synchronize()
    for i, out, ref in zip(VIEWS, outs, refs):
        got = out.cpu().numpy().reshape(H, W, 3)
        assert np.array_equal(got, ref), "%s: view %d differs from fvv_synthesize at %d px" % (
            case, i, int((got != ref).any(axis=-1).sum()))
        orc = oracle_mod.synthesize(cams, wl["rgb"], wl["depth"], wl["views"][i], wl["look_at"], **over)
        assert np.array_equal(got, orc["rgb"]), "%s: view %d differs from the oracle at %d px" % (
            case, i, int((got != orc["rgb"]).any(axis=-1).sum()))


def test_noalloc_leaves_free_device_memory_unchanged(arc):
    import torch
    F = lib()
    wl = arc
    cams = wl["cams"]
    H, W = cams[0].height, cams[0].width
    rig = F.rig(cams, wl["look_at"])
    dp, dps, rp, rps = _device_frames(wl)
    out = torch.zeros((H, W * 3), dtype=torch.uint8, device="cuda")
    F.fvv_synthesize_noalloc(rig, None, dp, dps, rp, rps, wl["views"][3], out, W * 3)   # warm-up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for i in (4, 5, 6):
        F.fvv_synthesize_noalloc(rig, None, dp, dps, rp, rps, wl["views"][i], out, W * 3)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, "free device memory changed by %d bytes" % (free0 - free1)


def test_noalloc_rejects_oversized_view_host_output_and_wide_pitch(arc):
    import torch
    F = lib()
    wl = arc
    cams = wl["cams"]
    K, W = len(cams), cams[0].width
    rig = F.rig(cams, wl["look_at"])
    dp, dps, rp, rps = _device_frames(wl)
    big = wl["views"][0].copy()
    big.width, big.height = 2048, 1025                      # one row over the limit
    out = torch.zeros((1025, 2048 * 3), dtype=torch.uint8, device="cuda")
    with pytest.raises(F.FvvError) as e:
        F.fvv_synthesize_noalloc(rig, None, dp, dps, rp, rps, big, out, 2048 * 3)
    assert e.value.code == F.FVV_ERR_INVALID_ARG
    assert str(F.FVV_NOALLOC_MAX_PIXELS) in F.fvv_last_error()
    host_out = np.zeros((720, W * 3), np.uint8)
    with pytest.raises(F.FvvError) as e:
        F.fvv_synthesize_noalloc(rig, None, dp, dps, rp, rps, wl["views"][0], host_out, W * 3)
    assert e.value.code == F.FVV_ERR_INVALID_ARG
    # a pitch whose last row would leave the 32-bit index range of a frame
    out = torch.zeros((720, W * 3), dtype=torch.uint8, device="cuda")
    with pytest.raises(F.FvvError) as e:
        F.fvv_synthesize_noalloc(rig, None, dp, [1 << 24] * K, rp, rps, wl["views"][0], out, W * 3)
    assert e.value.code == F.FVV_ERR_INVALID_ARG
    assert "pitch" in F.fvv_last_error()
