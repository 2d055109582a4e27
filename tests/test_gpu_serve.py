"""The continuous-batching serving loop (fvv_serve_*), on the GPU.

Many viewers submit viewpoint requests of mixed resolutions while batches
are running; every result must equal the same view synthesised alone
(fvv_synthesize) within the parity tolerance, and admission must honour the
pending limit and the memory budget."""
import time

import numpy as np
import pytest

import synthetic as S
from fvv_helpers import lib, psnr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rig_small():
    return S.workload("plain_9cam_1280x720", scale=0.25)        # 320 x 180 cameras


def _ctx_with_frames(F, wl, **opt):
    ctx = F.fvv_create(F.rig(wl["cams"], wl["look_at"]), F.fvv_default_options(**opt))
    H, W = wl["cams"][0].height, wl["cams"][0].width
    for k in range(len(wl["cams"])):
        F.fvv_upload_frame(ctx, k, np.ascontiguousarray(wl["rgb"][k]), W * 3,
                           np.ascontiguousarray(wl["depth"][k]), W * 2, 0)
    return ctx


def _view(base, W, H, f):
    v = base.copy()
    v.width, v.height, v.fx, v.fy, v.cx, v.cy = W, H, f, f, (W - 1) / 2, (H - 1) / 2
    return v


def test_serve_results_equal_alone_under_mixed_load(rig_small):
    import torch
    F = lib()
    wl = rig_small
    rng = np.random.default_rng(3)
    # 640x360 : 1280x720 : 1920x1080 = 2:1:1, large enough that requests queue
    # behind running batches and get packed together
    sizes = [(640, 360, 250.0), (640, 360, 250.0), (1280, 720, 500.0), (1920, 1080, 750.0)]
    reqs = []
    for i in range(48):
        W, H, f = sizes[rng.integers(0, 4)]
        reqs.append((i % 4, _view(wl["views"][int(rng.integers(0, 300))], W, H, f)))
    ctx = _ctx_with_frames(F, wl)
    try:
        F.fvv_serve_start(ctx, F.fvv_serve_default_cfg(lanes=3, max_batch=4,
                                                        memory_budget=512 << 20))
        outs, tickets = [], []
        for i, (viewer, v) in enumerate(reqs):
            if i % 3 == 0:       # every third output in host memory, the rest on the device
                outs.append(np.zeros((v.height, v.width * 3), np.uint8))
            else:
                outs.append(torch.zeros((v.height, v.width * 3), dtype=torch.uint8, device="cuda"))
        torch.cuda.synchronize()
        fv = [F.camera(v) for _, v in reqs]
        for i, ((viewer, v), o) in enumerate(zip(reqs, outs)):
            tickets.append(F.fvv_serve_submit(ctx, viewer, fv[i], o, v.width * 3))
            if i == 23:
                time.sleep(0.002)   # a second burst arrives while earlier batches run
        for t in tickets:
            F.fvv_serve_poll(ctx, t, 5_000_000)
        st = F.fvv_serve_stats(ctx)
        assert st["completed"] == 48 and st["failed"] == 0
        assert st["batches"] < 48 and st["mean_batch"] > 1.0
        assert st["p50_ms"] > 0 and st["p99_ms"] >= st["p50_ms"]
        F.fvv_serve_stop(ctx)
        for (viewer, v), o in zip(reqs, outs):
            ref = torch.zeros((v.height, v.width * 3), dtype=torch.uint8, device="cuda")
            F.fvv_synthesize(ctx, v, ref, v.width * 3)
            torch.cuda.synchronize()
            a = o.cpu().numpy() if hasattr(o, "cpu") else o
            b = ref.cpu().numpy()
            d = np.abs(a.astype(int) - b.astype(int)).reshape(v.height, v.width, 3)
            assert (d <= 1).all(axis=-1).mean() >= 0.999
            assert psnr(a, b) >= 50.0
            assert np.array_equal(a, b)      # the same kernels on the same inputs
    finally:
        F.fvv_destroy(ctx)


def test_serve_admission_and_errors(rig_small):
    import torch
    F = lib()
    wl = rig_small
    v = _view(wl["views"][10], 160, 90, 62.5)
    out = torch.zeros((90, 480), dtype=torch.uint8, device="cuda")
    # no frame yet: NOT_READY
    ctx = F.fvv_create(F.rig(wl["cams"], wl["look_at"]), F.fvv_default_options())
    try:
        F.fvv_serve_start(ctx, F.fvv_serve_default_cfg(lanes=1, max_batch=2, max_pending=3,
                                                        memory_budget=16 << 20))
        with pytest.raises(F.FvvError) as e:
            F.fvv_serve_submit(ctx, 0, v, out, 480)
        assert e.value.code == F.FVV_ERR_NOT_READY
        with pytest.raises(F.FvvError) as e:
            F.fvv_serve_start(ctx, None)
        assert e.value.code == F.FVV_ERR_STATE
        F.fvv_serve_stop(ctx)
    finally:
        F.fvv_destroy(ctx)
    ctx = _ctx_with_frames(F, wl)
    try:
        F.fvv_serve_start(ctx, F.fvv_serve_default_cfg(lanes=1, max_batch=2, max_pending=3,
                                                        memory_budget=16 << 20))
        ts = [F.fvv_serve_submit(ctx, 0, v, out, 480) for _ in range(3)]
        with pytest.raises(F.FvvError) as e:          # pending limit (tickets not polled)
            F.fvv_serve_submit(ctx, 0, v, out, 480)
        assert e.value.code == F.FVV_ERR_BUSY
        for t in ts:
            F.fvv_serve_poll(ctx, t, 5_000_000)
        with pytest.raises(F.FvvError) as e:          # collected already
            F.fvv_serve_poll(ctx, ts[0], 0)
        assert e.value.code == F.FVV_ERR_INVALID_ARG
        huge = _view(wl["views"][10], 4000, 3000, 1000.0)
        big_out = torch.zeros((3000, 12000), dtype=torch.uint8, device="cuda")
        with pytest.raises(F.FvvError) as e:          # larger than one lane's budget
            F.fvv_serve_submit(ctx, 0, huge, big_out, 12000)
        assert e.value.code == F.FVV_ERR_BUDGET
        with pytest.raises(F.FvvError) as e:
            F.fvv_serve_start(ctx, F.fvv_serve_default_cfg(lanes=0))
        assert e.value.code in (F.FVV_ERR_INVALID_ARG, F.FVV_ERR_STATE)
        F.fvv_serve_stop(ctx)
        with pytest.raises(F.FvvError) as e:
            F.fvv_serve_submit(ctx, 0, v, out, 480)
        assert e.value.code == F.FVV_ERR_STATE
    finally:
        F.fvv_destroy(ctx)


def test_serve_while_frames_update(rig_small):
    """Frames keep arriving (new ticks) while requests are served; every
    result equals the alone-result of one of the uploaded ticks."""
    import torch
    F = lib()
    wl = rig_small
    H, W = wl["cams"][0].height, wl["cams"][0].width
    wl2 = {"rgb": np.ascontiguousarray(wl["rgb"][:, :, ::-1]), "depth": wl["depth"]}
    frames = [(wl["rgb"], wl["depth"]), (wl2["rgb"], wl2["depth"])]
    v = _view(wl["views"][70], 320, 180, 125.0)
    ctx = _ctx_with_frames(F, wl, frame_slots=3)
    try:
        refs = []
        for t, (rgb, dep) in enumerate(frames):
            for k in range(len(wl["cams"])):
                F.fvv_upload_frame(ctx, k, np.ascontiguousarray(rgb[k]), W * 3,
                                   np.ascontiguousarray(dep[k]), W * 2, 10 + t)
            r = torch.zeros((180, 960), dtype=torch.uint8, device="cuda")
            F.fvv_synthesize(ctx, v, r, 960)
            torch.cuda.synchronize()
            refs.append(r.cpu().numpy())
        assert not np.array_equal(refs[0], refs[1])
        F.fvv_serve_start(ctx, F.fvv_serve_default_cfg(lanes=2, max_batch=3))
        outs, ts = [], []
        for i in range(24):
            if i % 4 == 0:
                rgb, dep = frames[(i // 4) % 2]
                for k in range(len(wl["cams"])):
                    F.fvv_upload_frame(ctx, k, np.ascontiguousarray(rgb[k]), W * 3,
                                       np.ascontiguousarray(dep[k]), W * 2, 12 + i // 4)
            o = torch.zeros((180, 960), dtype=torch.uint8, device="cuda")
            outs.append(o)
            ts.append(F.fvv_serve_submit(ctx, i % 3, v, o, 960))
        for t in ts:
            F.fvv_serve_poll(ctx, t, 5_000_000)
        F.fvv_serve_stop(ctx)
        for o in outs:
            a = o.cpu().numpy()
            assert np.array_equal(a, refs[0]) or np.array_equal(a, refs[1])
    finally:
        F.fvv_destroy(ctx)


@pytest.mark.parametrize("precision", ["bf16", "e4m3"])
def test_serve_refined_equals_alone(rig_small, precision):
    """Refinement on: requests of two sizes are served in same-size batches
    through the network; every result equals fvv_synthesize_refined of the
    view alone, byte for byte (the same kernels on the same inputs; no
    reduction in the forward pass depends on the batch)."""
    import torch
    F = lib()
    wl = rig_small
    rng = np.random.default_rng(11)
    sizes = [(320, 180, 125.0), (640, 360, 250.0)]
    reqs = []
    for i in range(20):
        W, H, f = sizes[int(rng.integers(0, 2))]
        reqs.append(_view(wl["views"][int(rng.integers(0, 300))], W, H, f))
    ctx = _ctx_with_frames(F, wl)
    try:
        with pytest.raises(F.FvvError) as e:                     # no network yet
            F.fvv_serve_start(ctx, F.fvv_serve_default_cfg(refine=1))
        assert e.value.code == F.FVV_ERR_STATE
        F.fvv_refine_init(ctx, None)
        if precision == "e4m3":
            F.fvv_refine_quantize(ctx, None, np.full(10, 0.02, np.float32))
        F.fvv_serve_start(ctx, F.fvv_serve_default_cfg(lanes=2, max_batch=4, memory_budget=128 << 20,
                                                        refine=1))
        probe = torch.zeros((180, 960), dtype=torch.uint8, device="cuda")
        with pytest.raises(F.FvvError) as e:                     # the network is in use
            F.fvv_synthesize_refined(ctx, reqs[0], probe, 960)
        assert e.value.code == F.FVV_ERR_BUSY
        with pytest.raises(F.FvvError) as e:
            F.fvv_refine_set_precision(ctx, F.FVV_PREC_BF16)
        assert e.value.code == F.FVV_ERR_BUSY
        with pytest.raises(F.FvvError) as e:                     # not a multiple of 4
            F.fvv_serve_submit(ctx, 0, _view(wl["views"][3], 322, 180, 125.0), probe, 966)
        assert e.value.code == F.FVV_ERR_INVALID_ARG
        outs = []
        for i, v in enumerate(reqs):
            if i % 3 == 0:
                outs.append(np.zeros((v.height, v.width * 3), np.uint8))
            else:
                outs.append(torch.zeros((v.height, v.width * 3), dtype=torch.uint8, device="cuda"))
        torch.cuda.synchronize()
        tickets = [F.fvv_serve_submit(ctx, i % 4, F.camera(v), o, v.width * 3)
                   for i, (v, o) in enumerate(zip(reqs, outs))]
        for t in tickets:
            F.fvv_serve_poll(ctx, t, 10_000_000)
        st = F.fvv_serve_stats(ctx)
        assert st["completed"] == 20 and st["failed"] == 0
        assert st["batches"] < 20
        F.fvv_serve_stop(ctx)
        changed = 0
        for v, o in zip(reqs, outs):
            ref = torch.zeros((v.height, v.width * 3), dtype=torch.uint8, device="cuda")
            F.fvv_synthesize_refined(ctx, v, ref, v.width * 3)
            plain = torch.zeros_like(ref)
            F.fvv_synthesize(ctx, v, plain, v.width * 3)
            torch.cuda.synchronize()
            a = o.cpu().numpy() if hasattr(o, "cpu") else o
            assert np.array_equal(a, ref.cpu().numpy())
            changed += int(not np.array_equal(a, plain.cpu().numpy()))
        assert changed == len(reqs)                              # the network did run
    finally:
        F.fvv_destroy(ctx)


# ---- persistent serving kernel ---------------------------------------------
def test_persistent_kernel_waits_run_out_cleanly(rig_small):
    """The persistent kernel's wait for work returns after its idle limit, and
    a grid barrier that cannot complete gives up after its limit and reports
    it; the CUDA context keeps working (a synthesis still matches)."""
    import torch
    F = lib()
    t0 = time.perf_counter()
    assert F.fvv_selftest_persistent_wait(False, 30000) == F.FVV_ERR_TIMEOUT
    assert "idle" in F.fvv_last_error()
    assert time.perf_counter() - t0 < 1.5
    t0 = time.perf_counter()
    assert F.fvv_selftest_persistent_wait(True, 40000) == F.FVV_ERR_TIMEOUT
    assert "barrier" in F.fvv_last_error()
    assert 0.03 <= time.perf_counter() - t0 < 1.5
    wl = rig_small
    ctx = _ctx_with_frames(F, wl)
    try:
        v = wl["views"][5]
        a = torch.zeros((v.height, v.width * 3), dtype=torch.uint8, device="cuda")
        F.fvv_synthesize(ctx, v, a, v.width * 3)
        torch.cuda.synchronize()
        assert int(a.float().sum().item()) > 0
    finally:
        F.fvv_destroy(ctx)


def test_persistent_serve_equals_alone_and_relaunches_after_idle(rig_small):
    """Mixed resolutions served through the persistent kernel equal the same
    views synthesised alone byte for byte; a request after the kernel went
    idle (and returned) relaunches it; an upload while batches run waits for
    the batches that read its slot."""
    import torch
    F = lib()
    wl = rig_small
    rng = np.random.default_rng(11)
    sizes = [(640, 360, 250.0), (640, 360, 250.0), (1280, 720, 500.0), (1920, 1080, 750.0)]
    reqs = []
    for i in range(40):
        W, H, f = sizes[rng.integers(0, 4)]
        reqs.append((i % 4, _view(wl["views"][int(rng.integers(0, 300))], W, H, f)))
    ctx = _ctx_with_frames(F, wl, frame_slots=2)
    H0, W0 = wl["cams"][0].height, wl["cams"][0].width
    try:
        F.fvv_serve_start(ctx, F.fvv_serve_default_cfg(lanes=3, max_batch=4, memory_budget=512 << 20,
                                                        persistent=1, max_width=1920, idle_us=20000))
        # a host output is refused in this mode
        with pytest.raises(F.FvvError) as e:
            F.fvv_serve_submit(ctx, 0, reqs[0][1], np.zeros((reqs[0][1].height, reqs[0][1].width * 3), np.uint8),
                               reqs[0][1].width * 3)
        assert e.value.code == F.FVV_ERR_INVALID_ARG
        outs = [torch.zeros((v.height, v.width * 3), dtype=torch.uint8, device="cuda") for _, v in reqs]
        torch.cuda.synchronize()
        tickets = []
        for i, ((viewer, v), o) in enumerate(zip(reqs, outs)):
            tickets.append(F.fvv_serve_submit(ctx, viewer, v, o, v.width * 3))
            if i == 19:
                time.sleep(0.002)
        for t in tickets:
            F.fvv_serve_poll(ctx, t, 5_000_000)
        st = F.fvv_serve_stats(ctx)
        assert st["completed"] == 40 and st["failed"] == 0
        # idle longer than the kernel's limit: it returns; the next request relaunches it
        time.sleep(0.1)
        v = reqs[0][1]
        late = torch.zeros_like(outs[0])
        F.fvv_serve_poll(ctx, F.fvv_serve_submit(ctx, 9, v, late, v.width * 3), 5_000_000)
        assert torch.equal(late, outs[0])
        # uploads of new ticks into the two-slot ring while requests run
        more = []
        for k in range(6):
            for cam in range(len(wl["cams"])):
                F.fvv_upload_frame(ctx, cam, np.ascontiguousarray(wl["rgb"][cam]), W0 * 3,
                                   np.ascontiguousarray(wl["depth"][cam]), W0 * 2, 1 + k)
            o = torch.zeros_like(outs[k])
            more.append((o, F.fvv_serve_submit(ctx, k, reqs[k][1], o, reqs[k][1].width * 3)))
        for o, t in more:
            F.fvv_serve_poll(ctx, t, 5_000_000)
        F.fvv_serve_stop(ctx)
        for k, (o, _) in enumerate(more):          # the same frames in every tick: the same views
            assert torch.equal(o, outs[k])
        for (viewer, v), o in zip(reqs, outs):
            ref = torch.zeros((v.height, v.width * 3), dtype=torch.uint8, device="cuda")
            F.fvv_synthesize(ctx, v, ref, v.width * 3)
            torch.cuda.synchronize()
            assert torch.equal(o, ref)
    finally:
        F.fvv_destroy(ctx)


@pytest.mark.parametrize("persistent", [0, 1])
def test_batch_window_coalesces_sparse_requests(rig_small, persistent):
    """Requests 1 ms apart find the GPU idle, so without a window every batch
    holds one view; with a 40 ms window they leave together.  The results
    still equal the views rendered alone, and no request waits much beyond
    the window."""
    import torch
    F = lib()
    wl = rig_small
    views = [_view(wl["views"][17 * i], 320, 180, 125.0) for i in range(12)]
    ctx = _ctx_with_frames(F, wl)
    try:
        stats = {}
        for window in (0, 40_000):
            F.fvv_serve_start(ctx, F.fvv_serve_default_cfg(lanes=2, max_batch=16, batch_window_us=window,
                                                            persistent=persistent))
            outs = [torch.zeros((v.height, v.width * 3), dtype=torch.uint8, device="cuda") for v in views]
            torch.cuda.synchronize()
            tickets = []
            for i, (v, o) in enumerate(zip(views, outs)):
                tickets.append(F.fvv_serve_submit(ctx, i, F.camera(v), o, v.width * 3))
                time.sleep(0.001)
            for t in tickets:
                F.fvv_serve_poll(ctx, t, 5_000_000)
            stats[window] = F.fvv_serve_stats(ctx)
            F.fvv_serve_stop(ctx)
            for v, o in zip(views, outs):
                ref = torch.zeros_like(o)
                F.fvv_synthesize(ctx, v, ref, v.width * 3)
                torch.cuda.synchronize()
                assert torch.equal(o, ref)
        assert stats[0]["completed"] == 12 and stats[40_000]["completed"] == 12
        assert stats[40_000]["mean_batch"] >= 4.0 > stats[0]["mean_batch"]
        assert stats[40_000]["max_ms"] < 40.0 + 200.0
    finally:
        F.fvv_destroy(ctx)


def test_batch_window_is_bounded(rig_small):
    F = lib()
    ctx = _ctx_with_frames(F, rig_small)
    try:
        with pytest.raises(F.FvvError) as e:
            F.fvv_serve_start(ctx, F.fvv_serve_default_cfg(batch_window_us=2_000_000))
        assert e.value.code == F.FVV_ERR_INVALID_ARG
    finally:
        F.fvv_destroy(ctx)
