"""The depth codec (Sec. IV-A, V-A, Eq. (1)-(3)) on the GPU against the oracle
(oracle/codec.py): encoding, decoding and the fused YUV upload are integer
work decided by tables both sides build in FP64, so every byte and every
depth code must match exactly."""
import numpy as np
import pytest

import synthetic as S
from oracle import codec as K
from fvv_helpers import lib

pytestmark = pytest.mark.gpu

CODEC = dict(z_near=0.4, z_far=6.0, alpha=0.004, beta=0.995)


@pytest.fixture(scope="module")
def setup():
    F = lib()
    wl = S.workload("plain_9cam_1280x720", scale=0.25)              # 320 x 180 cameras
    ctx = F.fvv_create(F.rig(wl["cams"], wl["look_at"]))
    for k in range(len(wl["cams"])):
        F.fvv_set_depth_codec(ctx, k, F.fvv_depth_codec_default(**CODEC))
    yield F, ctx, wl
    F.fvv_destroy(ctx)


def _depth_cases(wl):
    """The workload's depth (noise, dropouts) plus codes out of range and
    background-signalled rows."""
    d = np.array(wl["depth"][0], np.uint16)
    d[:4, :] = 65534                                   # beyond z_far
    d[4:8, :] = 100                                    # nearer than z_near
    d[8:10, :] = 0                                     # no depth
    d[10:12, 3:] = 65535                               # background
    return d


def _planes(H, W):
    import torch
    return (torch.zeros((H, W), dtype=torch.uint8, device="cuda"),
            torch.zeros((H // 2, W // 2), dtype=torch.uint8, device="cuda"),
            torch.zeros((H // 2, W // 2), dtype=torch.uint8, device="cuda"))


def test_encode_matches_oracle(setup):
    import torch
    F, ctx, wl = setup
    H, W = wl["depth"][0].shape
    d = _depth_cases(wl)
    y, u, v = _planes(H, W)
    F.fvv_depth_encode_yuv(ctx, 0, torch.from_numpy(d.astype(np.int16)).cuda(), W * 2, y, W, u, v, W // 2)
    torch.cuda.synchronize()
    ry, ru, rv = K.encode(d, unit_m=0.001, **CODEC)
    assert np.array_equal(y.cpu().numpy(), ry)
    assert np.array_equal(u.cpu().numpy(), ru)
    assert np.array_equal(v.cpu().numpy(), rv)


def test_decode_matches_oracle_on_every_code(setup):
    """Random planes: every 12-bit code at every block position occurs."""
    import torch
    F, ctx, wl = setup
    H, W = wl["depth"][0].shape
    rng = np.random.default_rng(4)
    Y = rng.integers(0, 256, (H, W), dtype=np.uint8)
    U = rng.integers(0, 256, (H // 2, W // 2), dtype=np.uint8)
    V = rng.integers(0, 256, (H // 2, W // 2), dtype=np.uint8)
    out = torch.zeros((H, W), dtype=torch.int16, device="cuda")
    F.fvv_depth_decode_yuv(ctx, 3, torch.from_numpy(Y).cuda(), W, torch.from_numpy(U).cuda(),
                           torch.from_numpy(V).cuda(), W // 2, out, W * 2)
    torch.cuda.synchronize()
    ref = K.decode(Y, U, V, CODEC["z_near"], CODEC["z_far"], 0.001)
    assert np.array_equal(out.cpu().numpy().view(np.uint16), ref)
    assert len(np.unique(K.unpack_yuv420(Y, U, V))) > 4000


@pytest.mark.parametrize("host", [False, True])
def test_yuv_upload_synthesises_like_the_decoded_depth(setup, oracle_mod, host):
    """Frames uploaded as YUV420 depth give the same z-buffer keys as the
    oracle run on the oracle-decoded depth."""
    import torch
    F, ctx0, wl = setup
    cams = wl["cams"]
    H, W = cams[0].height, cams[0].width
    ctx = F.fvv_create(F.rig(cams, wl["look_at"]))
    try:
        dec = []
        for k in range(len(cams)):
            F.fvv_set_depth_codec(ctx, k, F.fvv_depth_codec_default(**CODEC))
            ry, ru, rv = K.encode(np.asarray(wl["depth"][k]), unit_m=0.001, **CODEC)
            dec.append(K.decode(ry, ru, rv, CODEC["z_near"], CODEC["z_far"], 0.001))
            planes = (ry, ru, rv) if host else tuple(torch.from_numpy(p).cuda() for p in (ry, ru, rv))
            F.fvv_upload_frame_yuv(ctx, k, np.ascontiguousarray(wl["rgb"][k]), W * 3, planes[0], W, planes[1],
                                   planes[2], W // 2, 0)
        v = wl["views"][17]
        keys = torch.zeros((H, W), dtype=torch.int64, device="cuda")
        out = torch.zeros((H, W * 3), dtype=torch.uint8, device="cuda")
        F.fvv_synthesize(ctx, v, out, W * 3, F.aux(keys=keys))
        torch.cuda.synchronize()
        ref = oracle_mod.synthesize(cams, wl["rgb"], np.stack(dec), v, wl["look_at"])
        assert np.array_equal(keys.cpu().numpy().view(np.uint64), ref["keys"])
        diff = np.abs(out.cpu().numpy().reshape(H, W, 3).astype(int) - ref["rgb"].astype(int))
        assert np.mean(diff <= 1) >= 0.999
    finally:
        F.fvv_destroy(ctx)


def test_codec_errors(setup):
    import torch
    F, ctx0, wl = setup
    cams = wl["cams"]
    ctx = F.fvv_create(F.rig(cams, wl["look_at"]))
    try:
        H, W = cams[0].height, cams[0].width
        y, u, v = _planes(H, W)
        d = torch.zeros((H, W), dtype=torch.int16, device="cuda")
        with pytest.raises(F.FvvError) as e:                      # no codec set yet
            F.fvv_depth_encode_yuv(ctx, 0, d, W * 2, y, W, u, v, W // 2)
        assert e.value.code == F.FVV_ERR_STATE
        with pytest.raises(F.FvvError) as e:
            F.fvv_set_depth_codec(ctx, 0, F.fvv_depth_codec_default(z_near=2.0, z_far=1.0))
        assert e.value.code == F.FVV_ERR_INVALID_ARG
        F.fvv_set_depth_codec(ctx, 0, F.fvv_depth_codec_default())
        with pytest.raises(F.FvvError) as e:                      # pitch too small
            F.fvv_depth_encode_yuv(ctx, 0, d, W, y, W, u, v, W // 2)
        assert e.value.code == F.FVV_ERR_INVALID_ARG
    finally:
        F.fvv_destroy(ctx)


@pytest.mark.parametrize("mode", ["host", "device", "jbf", "layered"])
def test_batched_yuv_tick_upload(setup, oracle_mod, mode):
    """A whole tick with YUV420 depth in one call (dense planar frames, all
    cameras): the z-buffer keys equal the oracle's on the oracle-decoded
    depth (pre-filtered with the filter on; with background codes in the
    layered form)."""
    import torch
    from oracle import jbf as J
    F, ctx0, wl = setup
    cams = wl["cams"]
    H, W = cams[0].height, cams[0].width
    lay = S.workload("layered_9cam_1280x720", scale=0.25) if mode == "layered" else None
    src = lay if lay is not None else wl
    opts = {"jbf": dict(jbf_radius=2), "layered": dict(layered=1)}.get(mode, {})
    ctx = F.fvv_create(F.rig(src["cams"], src["look_at"]), F.fvv_default_options(**opts))
    try:
        blocks, dec = [], []
        for k in range(len(cams)):
            F.fvv_set_depth_codec(ctx, k, F.fvv_depth_codec_default(**CODEC))
            if lay is not None:
                F.fvv_set_bg_depth(ctx, k, np.ascontiguousarray(lay["bg"][k]), W * 2)
            y, u, v = K.encode(np.asarray(src["depth"][k]), unit_m=0.001, **CODEC)
            blocks.append(np.concatenate([y.reshape(-1), u.reshape(-1), v.reshape(-1)]))
            dec.append(K.decode(y, u, v, CODEC["z_near"], CODEC["z_far"], 0.001))
        yuv = np.ascontiguousarray(np.stack(blocks))
        rgb = np.ascontiguousarray(src["rgb"])
        if mode == "device":
            yuv, rgb = torch.from_numpy(yuv).cuda(), torch.from_numpy(rgb).cuda()
        F.fvv_upload_frames_yuv(ctx, rgb, H * W * 3, W * 3, yuv, blocks[0].size, 0)
        dec = np.stack(dec)
        if mode == "jbf":
            dec = np.stack([J.jbf(dec[k], src["rgb"][k], radius=2) for k in range(len(cams))])
        v = src["views"][33]
        keys = torch.zeros((H, W), dtype=torch.int64, device="cuda")
        out = torch.zeros((H, W * 3), dtype=torch.uint8, device="cuda")
        F.fvv_synthesize(ctx, v, out, W * 3, F.aux(keys=keys))
        torch.cuda.synchronize()
        if lay is not None:
            ref = oracle_mod.synthesize_layered(src["cams"], src["rgb"], dec, lay["bg"], v, src["look_at"])
        else:
            ref = oracle_mod.synthesize(src["cams"], src["rgb"], dec, v, src["look_at"])
        assert np.array_equal(keys.cpu().numpy().view(np.uint64), ref["keys"])
        d = np.abs(out.cpu().numpy().reshape(H, W, 3).astype(int) - ref["rgb"].astype(int))
        assert (d <= 1).all(axis=-1).mean() >= 0.999
    finally:
        F.fvv_destroy(ctx)


@pytest.mark.parametrize("width,height,pad", [(320, 180, 0), (336, 40, 64), (330, 18, 0), (320, 20, 4)])
def test_decode_tick_in_one_call(width, height, pad):
    """fvv_depth_decode_yuv_frames over four cameras of one tick equals the
    oracle's decode of each frame: the 16-byte form (width a multiple of 16,
    aligned strides; also with padded depth rows) and the frame-by-frame
    form (width 330, or a depth pitch that is not a multiple of 16)."""
    import torch
    F = lib()
    base = S.workload("plain_2cam_320x240")["cams"][0]
    cams = []
    for k in range(4):
        c = base.copy()
        c.width, c.height = width, height
        c.t = c.t + np.array([0.05 * k, 0.0, 0.0])
        cams.append(c)
    ctx = F.fvv_create(F.rig(cams, np.zeros(3)))
    try:
        codecs = [dict(z_near=0.3 + 0.1 * k, z_far=6.0 + k, alpha=0.0, beta=1.0) for k in range(4)]
        for k in range(4):
            F.fvv_set_depth_codec(ctx, k, F.fvv_depth_codec_default(**codecs[k]))
        rng = np.random.default_rng(width + height + pad)
        H, W = height, width
        frame = H * W + 2 * (H // 2) * (W // 2)
        stride = (frame + 15) // 16 * 16
        yuv = rng.integers(0, 256, (4, stride), dtype=np.uint8)
        pitch = W * 2 + pad
        out = torch.full((4, H, pitch // 2), -7, dtype=torch.int16, device="cuda")
        F.fvv_depth_decode_yuv_frames(ctx, 4, torch.from_numpy(yuv).cuda(), stride, out, H * pitch, pitch)
        torch.cuda.synchronize()
        got = out.cpu().numpy().view(np.uint16)
        for k in range(4):
            b = yuv[k]
            Y = b[:H * W].reshape(H, W)
            U = b[H * W:H * W + (H // 2) * (W // 2)].reshape(H // 2, W // 2)
            V = b[H * W + (H // 2) * (W // 2):frame].reshape(H // 2, W // 2)
            ref = K.decode(Y, U, V, codecs[k]["z_near"], codecs[k]["z_far"], 0.001)
            assert np.array_equal(got[k, :, :W], ref), k
            assert (got[k, :, W:] == np.uint16(0xFFF9)).all()              # padding untouched
    finally:
        F.fvv_destroy(ctx)


def test_decode_tick_errors(setup):
    import torch
    F, ctx, wl = setup
    H, W = wl["depth"][0].shape
    frame = H * W + 2 * (H // 2) * (W // 2)
    yuv = torch.zeros((9, frame), dtype=torch.uint8, device="cuda")
    out = torch.zeros((9, H, W), dtype=torch.int16, device="cuda")
    for args in ((0, yuv, frame, out, H * W * 2, W * 2),          # no camera
                 (10, yuv, frame, out, H * W * 2, W * 2),         # more cameras than the rig
                 (9, yuv, frame - 1, out, H * W * 2, W * 2),      # overlapping frames
                 (9, yuv, frame, out, H * W * 2, W * 2 - 2),      # pitch too small
                 (9, yuv.cpu(), frame, out, H * W * 2, W * 2)):   # host memory
        with pytest.raises(F.FvvError) as e:
            F.fvv_depth_decode_yuv_frames(ctx, *args)
        assert e.value.code == F.FVV_ERR_INVALID_ARG
