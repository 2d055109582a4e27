"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the
same seeded inputs.  Keys, hole mask and depth bit-exact; colour within 1/255
on >= 99.9 % of pixels at >= 50 dB (see fvv_helpers.assert_parity)."""
import numpy as np
import pytest

import synthetic as S
from fvv_helpers import KEY_EMPTY, assert_parity, gpu_run, lib

pytestmark = pytest.mark.gpu


def _oracle(oracle_mod, cams, rgb, dep, view, O, **kw):
    return oracle_mod.synthesize(cams, rgb, dep, view, O, **kw)


def _opts(**kw):
    return lib().fvv_default_options(**kw)


def test_two_camera_plane_and_spheres(oracle_mod):
    """Two parallel cameras 320x240, f = 300 px, 100 mm baseline; the view
    midway between them."""
    wl = S.workload("plain_2cam_320x240")
    g = gpu_run(wl["cams"], wl["rgb"], wl["depth"], wl["views"], wl["look_at"])[0]
    ref = _oracle(oracle_mod, wl["cams"], wl["rgb"], wl["depth"], wl["views"][0], wl["look_at"])
    info = assert_parity(g, ref, "2cam")
    assert info["exact_rgb_fraction"] == 1.0


@pytest.fixture(scope="module")
def arc_small():
    return S.workload("plain_9cam_1280x720", scale=0.26)      # 333 x 187: ragged rows


@pytest.fixture(scope="module")
def arc_full():
    return S.workload("plain_9cam_1280x720")


def test_nine_camera_arc_small_batch(oracle_mod, arc_small):
    """Nine noisy cameras on the 90 deg arc, three views of the swing
    trajectory in one batch; 333 x 187 spans many tiles and a ragged tail."""
    wl = arc_small
    views = [wl["views"][i] for i in (0, 75, 210)]
    gs = gpu_run(wl["cams"], wl["rgb"], wl["depth"], views, wl["look_at"])
    for i, (g, v) in enumerate(zip(gs, views)):
        ref = _oracle(oracle_mod, wl["cams"], wl["rgb"], wl["depth"], v, wl["look_at"])
        assert_parity(g, ref, "view %d" % i)


def test_nine_camera_arc_full_size(oracle_mod, arc_full):
    """The 1280x720 nine-camera workload at full size, compared on every pixel."""
    wl = arc_full
    views = [wl["views"][i] for i in (37, 150)]
    gs = gpu_run(wl["cams"], wl["rgb"], wl["depth"], views, wl["look_at"])
    for i, (g, v) in enumerate(zip(gs, views)):
        ref = _oracle(oracle_mod, wl["cams"], wl["rgb"], wl["depth"], v, wl["look_at"])
        info = assert_parity(g, ref, "full view %d" % i)
        assert info["exact_rgb_fraction"] >= 0.999


@pytest.mark.parametrize("kw", [dict(n_ref=3), dict(n_ref=1), dict(crack_filter=0),
                                dict(hole_fill=0), dict(crack_filter=0, hole_fill=0, n_ref=2),
                                dict(tau_vis=0.0), dict(d_lo=1500, d_hi=3000), dict(pixel_weights=1),
                                dict(pixel_weights=1, n_ref=3, crack_filter=0), dict(z_min=1200.0)])
def test_options(oracle_mod, arc_small, kw):
    wl = arc_small
    v = wl["views"][40]
    g = gpu_run(wl["cams"], wl["rgb"], wl["depth"], [v], wl["look_at"], opts=_opts(**kw))[0]
    ref = _oracle(oracle_mod, wl["cams"], wl["rgb"], wl["depth"], v, wl["look_at"], **kw)
    assert_parity(g, ref, str(kw))


@pytest.mark.parametrize("z_min", [0.0, 1800.0])
def test_cameras_at_other_depths(oracle_mod, z_min):
    """Camera 1 0.4 m nearer a plane at 2 m than camera 0 and the view: a
    point lies 1600 mm from camera 1 and 2000 mm from the view, so the
    visibility test must use the depth in camera 1, and with z_min = 1800 mm
    camera 1's back-projections are rejected while both cameras splat."""
    W, H, f = 96, 64, 120.0
    cams = [S.Camera(W, H, f, f, (W - 1) / 2, (H - 1) / 2, np.eye(3), -np.array(c))
            for c in ((0.0, 0.0, 0.0), (0.05, 0.0, 0.4))]
    view = S.Camera(W, H, f, f, (W - 1) / 2, (H - 1) / 2, np.eye(3), -np.array([0.02, 0.0, 0.0]))
    rgb = np.stack([np.full((H, W, 3), c, np.uint8) for c in ((200, 20, 40), (10, 100, 250))])
    dep = np.stack([np.full((H, W), 2000, np.uint16), np.full((H, W), 1600, np.uint16)])
    g = gpu_run(cams, rgb, dep, [view], [0, 0, 2.0], opts=_opts(z_min=z_min, hole_fill=0))[0]
    ref = _oracle(oracle_mod, cams, rgb, dep, view, [0, 0, 2.0], z_min=z_min, hole_fill=0)
    assert_parity(g, ref, "z_min %g" % z_min)
    two = (ref["top3"][16:48, 24:72, 1] > 0)
    assert two.all() if z_min == 0.0 else not two.any()


def test_non_square_source_pixels(oracle_mod):
    """Five arc cameras with pixels 1.2 times taller than wide and a view
    with pixels 0.9 times as tall: the composed maps scale each axis by its
    own focal length, on both sides of the warp and the back-projection."""
    cams = S.rig_arc(5, 60.0, 1.5, 200, 120, 160.0)
    for c in cams:
        c.fy = 1.2 * c.fx
    scene = S.scene_random_objects(21, n_objects=10)
    rgb, dep = S.frames_for(scene, cams, noise_seed=3)
    view = S.arc_view(9.0, 1.55, 200, 120, 170.0)
    view.fy = 0.9 * view.fx
    g = gpu_run(cams, rgb, dep, [view], [0, 0, 0])[0]
    ref = _oracle(oracle_mod, cams, rgb, dep, view, [0, 0, 0])
    assert_parity(g, ref, "non-square sources")
    assert (ref["hole"] == 0).mean() > 0.5


def test_depth_code_range_ends(oracle_mod):
    """Codes d_lo - 1, d_lo, d_hi, d_hi + 1 in camera 0 (only the middle two
    splat) and camera 1's fetched codes below d_lo (it does not
    contribute): the kernels' unsigned range tests against the oracle."""
    W, H, f = 96, 64, 120.0
    cams = [S.Camera(W, H, f, f, (W - 1) / 2, (H - 1) / 2, np.eye(3), -np.array(c))
            for c in ((0.0, 0.0, 0.0), (0.05, 0.0, 0.4))]
    view = S.Camera(W, H, f, f, (W - 1) / 2, (H - 1) / 2, np.eye(3), -np.array([0.02, 0.0, 0.0]))
    rgb = np.stack([np.full((H, W, 3), c, np.uint8) for c in ((200, 20, 40), (10, 100, 250))])
    dep = np.stack([np.full((H, W), 2000, np.uint16), np.full((H, W), 1600, np.uint16)])
    dep[0, 10, 20], dep[0, 10, 30], dep[0, 10, 40], dep[0, 10, 50] = 1699, 1700, 2100, 2101
    kw = dict(d_lo=1700, d_hi=2100, hole_fill=0)
    g = gpu_run(cams, rgb, dep, [view], [0, 0, 2.0], opts=_opts(**kw))[0]
    ref = _oracle(oracle_mod, cams, rgb, dep, view, [0, 0, 2.0], **kw)
    assert_parity(g, ref, "code range ends")


def test_empty_input_all_holes(oracle_mod):
    cams = S.rig_arc(3, 30.0, 1.5, 40, 30, 40.0)
    rgb = np.full((3, 30, 40, 3), 200, np.uint8)
    dep = np.zeros((3, 30, 40), np.uint16)
    v = S.arc_view(5.0, 1.5, 40, 30, 40.0)
    g = gpu_run(cams, rgb, dep, [v], [0, 0, 0])[0]
    assert np.all(g["keys_raw"] == KEY_EMPTY) and np.all(g["keys"] == KEY_EMPTY)
    assert np.all(g["hole"] == 1) and not g["rgb"].any() and not g["depth"].any()
    assert_parity(g, _oracle(oracle_mod, cams, rgb, dep, v, [0, 0, 0]), "empty")


def test_identity_pose_reproduces_input(arc_small):
    wl = arc_small
    k = 4
    g = gpu_run(wl["cams"], wl["rgb"], wl["depth"], [wl["cams"][k].copy()], wl["look_at"],
                opts=_opts(crack_filter=0, hole_fill=0))[0]
    valid = wl["depth"][k] > 0
    assert np.array_equal(g["rgb"][valid], wl["rgb"][k][valid])
    assert np.array_equal(g["hole"].astype(bool), ~valid)


def test_host_outputs_and_padded_pitches(oracle_mod, arc_small):
    wl = arc_small
    v = wl["views"][120]
    ref = _oracle(oracle_mod, wl["cams"], wl["rgb"], wl["depth"], v, wl["look_at"])
    g = gpu_run(wl["cams"], wl["rgb"], wl["depth"], [v], wl["look_at"], host_out=True,
                rgb_pitch_pad=13, depth_pitch_pad=6, out_pitch_pad=5)[0]
    assert_parity(g, ref, "host outputs")


def test_mixed_view_sizes_in_one_batch(oracle_mod, arc_small):
    wl = arc_small
    base = wl["views"][60]
    views = []
    for (W, H, f) in ((1, 1, 3.0), (64, 48, 60.0), (333, 187, 260.0), (500, 260, 400.0)):
        c = base.copy()
        c.width, c.height, c.fx, c.fy, c.cx, c.cy = W, H, f, f, (W - 1) / 2, (H - 1) / 2
        views.append(c)
    gs = gpu_run(wl["cams"], wl["rgb"], wl["depth"], views, wl["look_at"])
    for g, v in zip(gs, views):
        assert_parity(g, _oracle(oracle_mod, wl["cams"], wl["rgb"], wl["depth"], v, wl["look_at"]),
                      "%dx%d" % (v.width, v.height))


def test_widest_views(oracle_mod, arc_small):
    """The resolve stages key rows in shared memory, so the view width is
    bounded by the per-CTA limit: a 5000-pixel-wide view (about 205 KB of
    shared memory at nine cameras) matches the oracle, and an 8192-wide one is
    refused as too wide before anything is launched."""
    import torch
    wl = arc_small
    base = wl["views"][120]
    wide = base.copy()
    W, H, f = 5000, 6, 260.0
    wide.width, wide.height, wide.fx, wide.fy, wide.cx, wide.cy = W, H, f, f, (W - 1) / 2, (H - 1) / 2
    g = gpu_run(wl["cams"], wl["rgb"], wl["depth"], [wide], wl["look_at"])[0]
    ref = _oracle(oracle_mod, wl["cams"], wl["rgb"], wl["depth"], wide, wl["look_at"])
    assert_parity(g, ref, "5000 wide")
    assert (ref["hole"] == 0).any() and (ref["hole"] == 1).any()
    F = lib()
    too = base.copy()
    too.width, too.height, too.fx, too.fy, too.cx, too.cy = 8192, 2, f, f, 4095.5, 0.5
    ctx = F.fvv_create(F.rig(wl["cams"], wl["look_at"]), None)
    try:
        for k, c in enumerate(wl["cams"]):
            F.fvv_upload_frame(ctx, k, np.ascontiguousarray(wl["rgb"][k]), c.width * 3,
                               np.ascontiguousarray(wl["depth"][k]), c.width * 2, 0)
        out = torch.zeros((2, 8192 * 3), dtype=torch.uint8, device="cuda")
        with pytest.raises(F.FvvError) as e:
            F.fvv_synthesize_batch(ctx, [too], [0], [out], [8192 * 3])
        assert e.value.code == F.FVV_ERR_INVALID_ARG
        assert "width" in str(e.value)
    finally:
        F.fvv_destroy(ctx)


@pytest.mark.parametrize("pixel_weights", [0, 1])
def test_non_square_view_pixels(oracle_mod, pixel_weights):
    """A view whose pixels are 1.3 times taller than wide (fy = 1.3 fx), 15
    mm from one camera and 585 mm from the other, over a plane at 1.5 m:
    the warp's maps and the per-pixel weights' (x - cx) / fx, (y - cy) / fy
    scale each axis by its own focal length."""
    W, H, f = 160, 120, 150.0
    cams = [S.Camera(W, H, f, f, (W - 1) / 2, (H - 1) / 2, np.eye(3), -np.array([x, 0.0, 0.0]))
            for x in (0.0, 0.6)]
    view = S.Camera(W, H, f, 1.3 * f, (W - 1) / 2, (H - 1) / 2, np.eye(3), -np.array([0.015, 0.0, 0.0]))
    rgb, dep = S.frames_for(S.scene_fronto_plane(1.5), cams)
    O = [0.3, 0.0, 1.5]
    g = gpu_run(cams, rgb, dep, [view], O, opts=_opts(pixel_weights=pixel_weights))[0]
    ref = _oracle(oracle_mod, cams, rgb, dep, view, O, pixel_weights=pixel_weights)
    assert_parity(g, ref, "fy = 1.3 fx")
    assert (ref["top3"][..., 1] > 0).mean() > 0.3


def test_sixty_four_cameras(oracle_mod):
    """The 6-bit camera field at its limit: 64 cameras on a full circle."""
    cams = S.rig_arc(64, 354.375, 1.5, 24, 16, 20.0)
    scene = S.scene_random_objects(11, n_objects=12)
    rgb, dep = S.frames_for(scene, cams)
    v = S.arc_view(176.0, 1.4, 48, 32, 40.0)          # next to camera 63 (177.2 deg)
    g = gpu_run(cams, rgb, dep, [v], [0, 0, 0])[0]
    ref = _oracle(oracle_mod, cams, rgb, dep, v, [0, 0, 0])
    assert_parity(g, ref, "64 cams")
    z, cam, src = oracle_mod.key_fields(g["keys_raw"])
    assert cam.max() == 63


def test_largest_source_image(oracle_mod):
    """The 26-bit source-pixel field at its limit: one 8192 x 8192 camera."""
    W = H = 8192
    cam = S.Camera(W, H, 4000.0, 4000.0, (W - 1) / 2, (H - 1) / 2, np.eye(3), np.zeros(3))
    rng = np.random.default_rng(5)
    dep = np.zeros((1, H, W), np.uint16)
    rows = np.arange(H - 64, H)
    dep[0, rows, :] = rng.integers(1500, 2500, (64, W)).astype(np.uint16)
    rgb = np.zeros((1, H, W, 3), np.uint8)
    rgb[0, rows] = rng.integers(0, 256, (64, W, 3)).astype(np.uint8)
    view = S.Camera(256, 256, 125.0, 125.0, 127.5, 127.5, np.eye(3), np.zeros(3))
    g = gpu_run([cam], rgb, dep, [view], [0, 0, 2.0], opts=_opts(crack_filter=0))[0]
    ref = _oracle(oracle_mod, [cam], rgb, dep, view, [0, 0, 2.0], crack_filter=0)
    assert_parity(g, ref, "8192^2")
    z, c, src = oracle_mod.key_fields(g["keys_raw"])
    assert src.max() > (1 << 26) - 8192 * 4


def test_frame_ring_ticks_and_errors(oracle_mod):
    """Ticks live in slot tick % frame_slots; a view may name any resident
    complete tick; evicted or incomplete ticks and stale uploads are errors."""
    import torch
    F = lib()
    cams = S.rig_arc(3, 40.0, 1.5, 64, 40, 60.0)
    frames = []
    for t in range(4):
        rgb, dep = S.frames_for(S.scene_random_objects(100 + t, n_objects=6), cams, noise_seed=t)
        frames.append((rgb, dep))
    v = S.arc_view(7.0, 1.5, 64, 40, 60.0)
    ctx = F.fvv_create(F.rig(cams, [0, 0, 0]), F.fvv_default_options(frame_slots=2))
    try:
        with pytest.raises(F.FvvError) as e:
            F.fvv_latest_tick(ctx)
        assert e.value.code == F.FVV_ERR_NOT_READY
        for t, (rgb, dep) in enumerate(frames):
            for k in range(3):
                F.fvv_upload_frame(ctx, k, np.ascontiguousarray(rgb[k]), 64 * 3,
                                   np.ascontiguousarray(dep[k]), 64 * 2, t)
        assert F.fvv_latest_tick(ctx) == 3
        outs = [torch.zeros((40, 64 * 3), dtype=torch.uint8, device="cuda") for _ in range(2)]
        F.fvv_synthesize_batch(ctx, [v, v], [2, 3], outs, [192, 192])
        torch.cuda.synchronize()
        for t, o in zip((2, 3), outs):
            ref = oracle_mod.synthesize(cams, frames[t][0], frames[t][1], v, [0, 0, 0])
            assert np.abs(o.cpu().numpy().reshape(40, 64, 3).astype(int) - ref["rgb"]).max() <= 1
        with pytest.raises(F.FvvError) as e:
            F.fvv_synthesize_batch(ctx, [v], [1], outs[:1], [192])
        assert e.value.code == F.FVV_ERR_NOT_READY
        with pytest.raises(F.FvvError) as e:
            F.fvv_upload_frame(ctx, 0, np.ascontiguousarray(frames[0][0][0]), 192,
                               np.ascontiguousarray(frames[0][1][0]), 128, 1)
        assert e.value.code == F.FVV_ERR_STATE
        # a partial tick is not visible
        F.fvv_upload_frame(ctx, 0, np.ascontiguousarray(frames[0][0][0]), 192,
                           np.ascontiguousarray(frames[0][1][0]), 128, 4)
        assert F.fvv_latest_tick(ctx) == 3
        with pytest.raises(F.FvvError) as e:
            F.fvv_synthesize_batch(ctx, [v], [4], outs[:1], [192])
        assert e.value.code == F.FVV_ERR_NOT_READY
    finally:
        F.fvv_destroy(ctx)


def test_user_stream_and_determinism(oracle_mod, arc_small):
    import torch
    wl = arc_small
    v = wl["views"][200]
    s = torch.cuda.Stream()
    a = gpu_run(wl["cams"], wl["rgb"], wl["depth"], [v], wl["look_at"], stream=s)[0]
    b = gpu_run(wl["cams"], wl["rgb"], wl["depth"], [v], wl["look_at"])[0]
    for k in ("rgb", "keys", "keys_raw", "depth", "top3", "hole"):
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("where", ["host", "device"])
def test_batched_tick_upload(oracle_mod, where):
    """fvv_upload_frames (all cameras of one size in one launch, host frames
    through one bulk copy each for colour and depth) gives the same frames as
    per-camera uploads: keys bit-exact with the oracle."""
    import torch
    F = lib()
    wl = S.workload("plain_9cam_1280x720", scale=0.25)
    cams = wl["cams"]
    K, H, W = len(cams), cams[0].height, cams[0].width
    ctx = F.fvv_create(F.rig(cams, wl["look_at"]), F.fvv_default_options(frame_slots=3))
    try:
        # padded rows and a gap between cameras exercise the strides
        rp, dp = W * 3 + 32, W * 2 + 64
        rcs, dcs = H * rp + 4096, H * dp + 2048
        rgb = np.zeros(K * rcs, np.uint8)
        dep = np.zeros(K * dcs, np.uint8)
        for k in range(K):
            for y in range(H):
                rgb[k * rcs + y * rp: k * rcs + y * rp + W * 3] = np.asarray(wl["rgb"][k][y]).reshape(-1)
                dep[k * dcs + y * dp: k * dcs + y * dp + W * 2] = np.asarray(wl["depth"][k][y], np.uint16).view(np.uint8)
        if where == "device":
            rgb, dep = torch.from_numpy(rgb).cuda(), torch.from_numpy(dep).cuda()
        for t in range(4):                       # several ticks through a 3-slot ring
            F.fvv_upload_frames(ctx, rgb, rcs, rp, dep, dcs, dp, t)
        v = wl["views"][5]
        keys = torch.zeros((H, W), dtype=torch.int64, device="cuda")
        out = torch.zeros((H, W * 3), dtype=torch.uint8, device="cuda")
        F.fvv_synthesize(ctx, v, out, W * 3, F.aux(keys=keys))
        torch.cuda.synchronize()
        ref = oracle_mod.synthesize(cams, wl["rgb"], wl["depth"], v, wl["look_at"])
        assert np.array_equal(keys.cpu().numpy().view(np.uint64), ref["keys"])
        diff = np.abs(out.cpu().numpy().reshape(H, W, 3).astype(int) - ref["rgb"].astype(int))
        assert np.mean(diff <= 1) >= 0.999
        assert F.fvv_latest_tick(ctx) == 3
    finally:
        F.fvv_destroy(ctx)
