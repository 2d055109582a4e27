"""The headline measurement's own launch configuration, checked against the
oracle: nine 1280x720 cameras, a 32-tick frame ring, batches of 32
1280x720 views each naming its own tick (two-row bands of the resolve), two
steps in a row on one context (the second runs on the z-buffer the first
resolve emptied, without a clear).  The ticks carry different colours, so a
view that read another tick's frames would fail."""
import numpy as np
import pytest

import synthetic as S
from fvv_helpers import lib, psnr

pytestmark = pytest.mark.gpu


def _tick_rgb(rgb, t):
    """Tick t's colour frames: the workload's, every channel shifted by 37 t."""
    return ((np.asarray(rgb, np.uint16) + 37 * (t % 4)) % 256).astype(np.uint8)


def test_bench_batches_match_the_oracle(oracle_mod):
    import torch
    F = lib()
    wl = S.workload("plain_9cam_1280x720")
    cams = wl["cams"]
    K, H, W = len(cams), cams[0].height, cams[0].width
    ctx = F.fvv_create(F.rig(cams, wl["look_at"]), F.fvv_default_options(frame_slots=32, max_batch=32))
    try:
        dep = torch.from_numpy(np.ascontiguousarray(np.stack(wl["depth"])).view(np.int16)).cuda()
        variants = [torch.from_numpy(np.ascontiguousarray(_tick_rgb(np.stack(wl["rgb"]), t))).cuda()
                    for t in range(4)]
        for t in range(32):
            F.fvv_upload_frames(ctx, variants[t % 4], H * W * 3, W * 3, dep, H * W * 2, W * 2, t)
        torch.cuda.synchronize()
        rng = np.random.default_rng(11)
        steps = [(list(rng.permutation(32)), list(rng.choice(300, 32, replace=False))) for _ in range(2)]
        for s, (ticks, vi) in enumerate(steps):
            views = [wl["views"][int(i)] for i in vi]
            ticks = [int(t) for t in ticks]
            outs = [torch.zeros((H, W * 3), dtype=torch.uint8, device="cuda") for _ in views]
            got = [{"depth": torch.zeros((H, W), dtype=torch.float32, device="cuda"),
                    "hole": torch.zeros((H, W), dtype=torch.uint8, device="cuda"),
                    "keys": torch.zeros((H, W), dtype=torch.int64, device="cuda"),
                    "keys_raw": torch.zeros((H, W), dtype=torch.int64, device="cuda")} for _ in views]
            aux = [F.aux(g["depth"], g["hole"], None, g["keys"], g["keys_raw"]) for g in got]
            F.fvv_synthesize_batch(ctx, views, ticks, outs, [W * 3] * len(views), aux)
            torch.cuda.synchronize()
            for j, (v, t) in enumerate(zip(views, ticks)):
                ref = oracle_mod.synthesize(cams, _tick_rgb(wl["rgb"], t), wl["depth"], v, wl["look_at"])
                label = "step %d view %d (tick %d)" % (s, j, t)
                g = {k: x.cpu().numpy() for k, x in got[j].items()}
                assert np.array_equal(g["keys_raw"].view(np.uint64), ref["keys_raw"]), label
                assert np.array_equal(g["keys"].view(np.uint64), ref["keys"]), label
                assert np.array_equal(g["hole"], ref["hole"]), label
                assert np.array_equal(g["depth"], ref["depth"]), label
                rgb = outs[j].cpu().numpy().reshape(H, W, 3)
                d = np.abs(rgb.astype(int) - ref["rgb"].astype(int))
                assert (d <= 1).all(axis=-1).mean() >= 0.999, label
                assert psnr(rgb, ref["rgb"]) >= 50.0, label
                assert (d == 0).all(axis=-1).mean() >= 0.999, label
    finally:
        F.fvv_destroy(ctx)
