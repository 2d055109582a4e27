"""Consecutive batches on one context reuse its z-buffer scratch: a batch
whose layout (view sizes, in order) matches the previous one's splats into
the buffer that the previous resolve emptied, without a clear launch; any
other batch clears first.  Every batch, in every order of layouts, must
still match the oracle exactly (keys before and after the filter, holes,
depth) and within the colour bar."""
import numpy as np
import pytest

import synthetic as S
from fvv_helpers import lib, assert_parity

pytestmark = pytest.mark.gpu


def _view(base, W, H, f):
    v = base.copy()
    v.width, v.height, v.fx, v.fy, v.cx, v.cy = W, H, f, f, (W - 1) / 2, (H - 1) / 2
    return v


def _run_batch(F, ctx, views):
    import torch
    dev = torch.device("cuda")
    res, outs, pitches, auxs = [], [], [], []
    for v in views:
        H, W = v.height, v.width
        o = {"rgb_buf": torch.zeros((H, W * 3), dtype=torch.uint8, device=dev),
             "depth": torch.zeros((H, W), dtype=torch.float32, device=dev),
             "hole": torch.zeros((H, W), dtype=torch.uint8, device=dev),
             "top3": torch.zeros((H, W, 3), dtype=torch.float32, device=dev),
             "keys": torch.zeros((H, W), dtype=torch.int64, device=dev),
             "keys_raw": torch.zeros((H, W), dtype=torch.int64, device=dev)}
        outs.append(o["rgb_buf"])
        pitches.append(W * 3)
        auxs.append(F.aux(o["depth"], o["hole"], o["top3"], o["keys"], o["keys_raw"]))
        res.append(o)
    F.fvv_synthesize_batch(ctx, views, None, outs, pitches, auxs)
    torch.cuda.synchronize()
    out = []
    for v, o in zip(views, res):
        g = {k: x.cpu().numpy() for k, x in o.items()}
        g["rgb"] = g.pop("rgb_buf").reshape(v.height, v.width, 3)
        g["keys"] = g["keys"].view(np.uint64)
        g["keys_raw"] = g["keys_raw"].view(np.uint64)
        out.append(g)
    return out


def test_batches_reusing_the_scratch_match_the_oracle(oracle_mod):
    F = lib()
    wl = S.workload("plain_9cam_1280x720", scale=0.25)                # 320 x 180 cameras
    cams, H, W = wl["cams"], wl["cams"][0].height, wl["cams"][0].width
    ctx = F.fvv_create(F.rig(cams, wl["look_at"]))
    try:
        for k in range(len(cams)):
            F.fvv_upload_frame(ctx, k, np.ascontiguousarray(wl["rgb"][k]), W * 3,
                               np.ascontiguousarray(wl["depth"][k]), W * 2, 0)
        pose = iter(range(3, 300, 7))
        A = lambda: [wl["views"][next(pose)] for _ in range(4)]
        B = lambda: [wl["views"][next(pose)] for _ in range(2)]
        C = lambda: [_view(wl["views"][next(pose)], w, h, f) for w, h, f in
                     ((320, 180, 250.0), (160, 90, 125.0), (320, 180, 250.0), (200, 100, 150.0))]
        # A A A: two batches on emptied buffers; B then A: a changed layout
        # clears; C C: another layout; A last
        plan = [A, A, A, B, A, A, C, C, A]
        for i, make in enumerate(plan):
            views = make()
            got = _run_batch(F, ctx, views)
            for j, (v, g) in enumerate(zip(views, got)):
                ref = oracle_mod.synthesize(cams, wl["rgb"], wl["depth"], v, wl["look_at"])
                assert_parity(g, ref, "batch %d view %d" % (i, j))
    finally:
        F.fvv_destroy(ctx)
