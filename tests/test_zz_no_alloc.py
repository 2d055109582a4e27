"""The allocation-free entry point, fvv_synthesize_noalloc.

It serves callers that must not call cudaMalloc (a process whose device
memory belongs to another allocator, or a real-time render thread on which an
allocation would synchronise the device).  Its scratch is a fixed file-scope
device array.  These tests call it through the C ABI and check it against the
context-based fvv_synthesize on the same frames and views, with the tolerance
the parity tests use, for two calls in a row.  The file is collected last and
passes both alone in a fresh process and after the other tests.
"""
import numpy as np
import pytest

import synthetic as S
from fvv_helpers import lib, psnr

pytestmark = pytest.mark.gpu


def _device_frames(wl):
    """Frames in the library's device layout: uint16 depth, RGBA8 words."""
    import torch
    r = torch.from_numpy(np.ascontiguousarray(wl["rgb"])).cuda().to(torch.int32)
    rgba = (r[..., 0] | (r[..., 1] << 8) | (r[..., 2] << 16)).contiguous()
    depth = torch.from_numpy(np.ascontiguousarray(wl["depth"]).view(np.int16)).cuda().contiguous()
    return rgba, depth


@pytest.fixture(scope="module")
def arc():
    return S.workload("plain_9cam_1280x720")


def test_noalloc_matches_synthesize_two_calls_in_a_row(arc):
    import torch
    F = lib()
    wl = arc
    cams = wl["cams"]
    K, H, W = len(cams), cams[0].height, cams[0].width
    rig = F.rig(cams, wl["look_at"])
    opts = F.fvv_default_options()
    rgba, depth = _device_frames(wl)
    views = [wl["views"][37], wl["views"][150]]

    ctx = F.fvv_create(rig, opts)
    try:
        for k in range(K):
            F.fvv_upload_frame(ctx, k, np.ascontiguousarray(wl["rgb"][k]), W * 3,
                               np.ascontiguousarray(wl["depth"][k]), W * 2, 0)
        refs = []
        for v in views:
            ref = torch.zeros((H, W * 3), dtype=torch.uint8, device="cuda")
            F.fvv_synthesize(ctx, v, ref, W * 3)
            refs.append(ref)
        torch.cuda.synchronize()
    finally:
        F.fvv_destroy(ctx)

    for v, ref in zip(views, refs):            # two calls in a row, shared scratch
        out = torch.full((H, W * 3), 7, dtype=torch.uint8, device="cuda")
        F.fvv_synthesize_noalloc(rig, opts, [depth[k] for k in range(K)], [W * 2] * K,
                                 [rgba[k] for k in range(K)], [W * 4] * K, v, out, W * 3)
        torch.cuda.synchronize()
        a = out.cpu().numpy().reshape(H, W, 3).astype(int)
        b = ref.cpu().numpy().reshape(H, W, 3).astype(int)
        within = (np.abs(a - b) <= 1).all(axis=-1).mean()
        assert within >= 0.999, within
        assert psnr(a, b) >= 50.0


def test_noalloc_rejects_oversized_view_and_host_output(arc):
    import torch
    F = lib()
    wl = arc
    cams = wl["cams"]
    K, W = len(cams), cams[0].width
    rig = F.rig(cams, wl["look_at"])
    rgba, depth = _device_frames(wl)
    big = wl["views"][0].copy()
    big.width, big.height = 2048, 1025                      # one row over the limit
    out = torch.zeros((1025, 2048 * 3), dtype=torch.uint8, device="cuda")
    with pytest.raises(F.FvvError) as e:
        F.fvv_synthesize_noalloc(rig, None, [depth[k] for k in range(K)], [W * 2] * K,
                                 [rgba[k] for k in range(K)], [W * 4] * K, big, out, 2048 * 3)
    assert e.value.code == F.FVV_ERR_INVALID_ARG
    assert str(F.FVV_NOALLOC_MAX_PIXELS) in F.fvv_last_error()
    host_out = np.zeros((720, W * 3), np.uint8)
    with pytest.raises(F.FvvError) as e:
        F.fvv_synthesize_noalloc(rig, None, [depth[k] for k in range(K)], [W * 2] * K,
                                 [rgba[k] for k in range(K)], [W * 4] * K, wl["views"][0],
                                 host_out, W * 3)
    assert e.value.code == F.FVV_ERR_INVALID_ARG
