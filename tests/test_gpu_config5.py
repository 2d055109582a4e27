"""The stress configuration on the GPU: 18 cameras 1920x1080 on a 180 deg arc
of radius 2 m with the noise model of the 9-camera workload.  Full-size
views against the oracle on every pixel, and 64 viewers at mixed 720p/1080p
through the serving loop, every served view equal to the view rendered
alone."""
import numpy as np
import pytest

import synthetic as S
from fvv_helpers import assert_parity, gpu_run, lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def arc18():
    return S.workload("plain_18cam_1920x1080")


def test_eighteen_cameras_full_size(oracle_mod, arc18):
    wl = arc18
    views = [wl["views"][i] for i in (20, 180)]
    gs = gpu_run(wl["cams"], wl["rgb"], wl["depth"], views, wl["look_at"])
    for i, (g, v) in enumerate(zip(gs, views)):
        ref = oracle_mod.synthesize(wl["cams"], wl["rgb"], wl["depth"], v, wl["look_at"])
        info = assert_parity(g, ref, "18-camera 1080p view %d" % i)
        assert info["exact_rgb_fraction"] >= 0.999
        assert ref["hole"].mean() < 0.5


def test_sixty_four_viewers_mixed_resolutions(arc18):
    import torch
    F = lib()
    wl = arc18
    cams = wl["cams"]
    H, W = cams[0].height, cams[0].width
    ctx = F.fvv_create(F.rig(cams, wl["look_at"]), F.fvv_default_options(frame_slots=2, max_batch=16))
    try:
        F.fvv_upload_frames(ctx, np.ascontiguousarray(wl["rgb"]), H * W * 3, W * 3,
                            np.ascontiguousarray(wl["depth"]), H * W * 2, W * 2, 0)
        rng = np.random.default_rng(64)
        reqs = []
        for viewer in range(64):
            Wv, Hv, f = (1280, 720, 1000.0) if viewer % 2 == 0 else (1920, 1080, 1500.0)
            for _ in range(2):
                reqs.append((viewer, S.arc_view(float(rng.uniform(-80, 80)), 2.0, Wv, Hv, f)))
        F.fvv_serve_start(ctx, F.fvv_serve_default_cfg(lanes=3, max_batch=16, memory_budget=1 << 30))
        outs = [torch.zeros((v.height, v.width * 3), dtype=torch.uint8, device="cuda") for _, v in reqs]
        torch.cuda.synchronize()
        tickets = [F.fvv_serve_submit(ctx, viewer, F.camera(v), o, v.width * 3)
                   for (viewer, v), o in zip(reqs, outs)]
        for t in tickets:
            F.fvv_serve_poll(ctx, t, 20_000_000)
        st = F.fvv_serve_stats(ctx)
        assert st["completed"] == len(reqs) and st["failed"] == 0
        assert st["mean_batch"] > 1.0 and st["p99_ms"] >= st["p50_ms"] > 0
        F.fvv_serve_stop(ctx)
        for (viewer, v), o in zip(reqs[::7], outs[::7]):
            ref = torch.zeros_like(o)
            F.fvv_synthesize(ctx, v, ref, v.width * 3)
            torch.cuda.synchronize()
            assert torch.equal(o, ref)
    finally:
        F.fvv_destroy(ctx)
