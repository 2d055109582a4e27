"""The joint bilateral depth pre-filter (Sec. VI) on the GPU against the
oracle (oracle/jbf.py).  Every weight, sum and division is the same FP32
operation sequence on both sides, so the filtered codes must match exactly;
uploads with the filter on must synthesise like the oracle on the
oracle-filtered frames."""
import numpy as np
import pytest

import synthetic as S
from oracle import codec as K
from oracle import jbf as J
from fvv_helpers import lib

pytestmark = pytest.mark.gpu


def f32(x):
    """The value a float option field holds (the oracle gets the same)."""
    return float(np.float32(x))


@pytest.fixture(scope="module")
def arc():
    return S.workload("plain_9cam_1280x720", scale=0.26)          # 333 x 187


def _run(F, rgb, depth, **kw):
    import torch
    H, W = depth.shape
    o = F.fvv_default_options(**kw)
    r = torch.from_numpy(np.ascontiguousarray(rgb)).cuda()
    d = torch.from_numpy(np.ascontiguousarray(depth).view(np.int16)).cuda()
    out = torch.full((H, W), -1, dtype=torch.int16, device="cuda")
    F.fvv_depth_jbf(r, W * 3, d, W * 2, out, W * 2, W, H, o)
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint16)


@pytest.mark.parametrize("kw", [dict(jbf_radius=3),
                                dict(jbf_radius=5, jbf_sigma_s=3.3, jbf_sigma_c=17.5, jbf_min_valid=1),
                                dict(jbf_radius=7, jbf_sigma_s=6.0, jbf_sigma_c=4.0, jbf_min_valid=20),
                                dict(jbf_radius=1, jbf_min_valid=8, d_lo=1200, d_hi=3000)])
def test_filter_matches_oracle(arc, kw):
    F = lib()
    o = F.fvv_default_options(**kw)
    filled = 0
    for k in (0, 4, 8):
        got = _run(F, arc["rgb"][k], arc["depth"][k], **kw)
        ref = J.jbf(arc["depth"][k], arc["rgb"][k], radius=o.jbf_radius, sigma_s=f32(o.jbf_sigma_s),
                    sigma_c=f32(o.jbf_sigma_c), d_lo=o.d_lo, d_hi=o.d_hi, min_valid=o.jbf_min_valid)
        assert np.array_equal(got, ref), "camera %d: %d codes differ" % (k, int((got != ref).sum()))
        filled += int((got != arc["depth"][k]).sum())
    if o.jbf_min_valid < 8:                  # the 3x3 case with 8 valid neighbours may fill nothing
        assert filled > 0


def test_filter_edge_cases():
    """Tiny and one-row frames, no sources at all, background-signalled
    pixels (never sources, never filled)."""
    F = lib()
    rng = np.random.default_rng(3)
    for H, W in ((1, 1), (1, 17), (5, 3), (37, 1)):
        d = rng.integers(0, 4000, (H, W)).astype(np.uint16)
        d[rng.random((H, W)) < 0.4] = 0
        rgb = rng.integers(0, 256, (H, W, 3)).astype(np.uint8)
        got = _run(F, rgb, d, jbf_radius=2, jbf_min_valid=1)
        assert np.array_equal(got, J.jbf(d, rgb, radius=2, min_valid=1))
    z = np.zeros((20, 30), np.uint16)
    assert not _run(F, np.zeros((20, 30, 3), np.uint8), z, jbf_radius=3).any()
    lay = S.workload("layered_9cam_1280x720", scale=0.25)
    d, rgb = lay["depth"][2], lay["rgb"][2]
    got = _run(F, rgb, d, jbf_radius=3)
    assert np.array_equal(got, J.jbf(d, rgb, radius=3))
    assert np.array_equal(got == J.DEPTH_BG, d == J.DEPTH_BG)


@pytest.mark.parametrize("path", ["one_host", "one_device", "all_host", "all_device", "yuv"])
def test_uploads_with_the_filter_synthesise_like_the_filtered_frames(oracle_mod, arc, path):
    """Every upload path filters on the way into the frame ring: the
    z-buffer keys equal the oracle's on the oracle-filtered depth."""
    import torch
    F = lib()
    cams, rgb, dep = arc["cams"], arc["rgb"], arc["depth"]
    Kc, H, W = len(cams), cams[0].height, cams[0].width
    if path == "yuv":                                    # the codec needs even sizes
        H, W = H - H % 2, W - W % 2
        cams = [c.copy() for c in cams]
        for c in cams:
            c.width, c.height = W, H
        rgb = np.ascontiguousarray(rgb[:, :H, :W])
        dep = np.ascontiguousarray(dep[:, :H, :W])
    ctx = F.fvv_create(F.rig(cams, arc["look_at"]), F.fvv_default_options(jbf_radius=3))
    try:
        src = dep
        if path == "yuv":
            codec = dict(z_near=0.3, z_far=8.0, alpha=0.0, beta=1.0)
            dec = []
            for k in range(Kc):
                F.fvv_set_depth_codec(ctx, k, F.fvv_depth_codec_default(**codec))
                y, u, v = K.encode(dep[k], unit_m=0.001, **codec)
                dec.append(K.decode(y, u, v, codec["z_near"], codec["z_far"], 0.001))
                F.fvv_upload_frame_yuv(ctx, k, rgb[k], W * 3, y, W, u, v, W // 2, 0)
            src = np.stack(dec)
        elif path.startswith("one"):
            for k in range(Kc):
                r, d = np.ascontiguousarray(rgb[k]), np.ascontiguousarray(dep[k])
                if path == "one_device":
                    r = torch.from_numpy(r).cuda()
                    d = torch.from_numpy(d.view(np.int16)).cuda()
                F.fvv_upload_frame(ctx, k, r, W * 3, d, W * 2, 0)
        else:
            r, d = np.ascontiguousarray(rgb), np.ascontiguousarray(dep)
            if path == "all_device":
                r = torch.from_numpy(r).cuda()
                d = torch.from_numpy(d.view(np.int16)).cuda()
            F.fvv_upload_frames(ctx, r, H * W * 3, W * 3, d, H * W * 2, W * 2, 0)
        filt = np.stack([J.jbf(src[k], rgb[k], radius=3) for k in range(Kc)])
        v = arc["views"][70].copy()
        v.width, v.height = W, H
        keys = torch.zeros((H, W), dtype=torch.int64, device="cuda")
        out = torch.zeros((H, W * 3), dtype=torch.uint8, device="cuda")
        F.fvv_synthesize(ctx, v, out, W * 3, F.aux(keys=keys))
        torch.cuda.synchronize()
        ref = oracle_mod.synthesize(cams, rgb, filt, v, arc["look_at"])
        assert np.array_equal(keys.cpu().numpy().view(np.uint64), ref["keys"])
        d = np.abs(out.cpu().numpy().reshape(H, W, 3).astype(int) - ref["rgb"].astype(int))
        assert (d <= 1).all(axis=-1).mean() >= 0.999
        st = F.fvv_profile_read(ctx)
        assert "jbf" in st
    finally:
        F.fvv_destroy(ctx)


def test_filter_errors():
    import torch
    F = lib()
    d = torch.zeros((8, 8), dtype=torch.int16, device="cuda")
    o = torch.zeros((8, 8), dtype=torch.int16, device="cuda")
    rgb = torch.zeros((8, 24), dtype=torch.uint8, device="cuda")
    bad = [dict(jbf_radius=0), dict(jbf_radius=8), dict(jbf_radius=2, jbf_sigma_s=0.0),
           dict(jbf_radius=2, jbf_min_valid=25), dict(jbf_radius=2, jbf_min_valid=0)]
    for kw in bad:
        with pytest.raises(F.FvvError) as e:
            F.fvv_depth_jbf(rgb, 24, d, 16, o, 16, 8, 8, F.fvv_default_options(**kw))
        assert e.value.code == F.FVV_ERR_INVALID_ARG
    ok = F.fvv_default_options(jbf_radius=2)
    with pytest.raises(F.FvvError) as e:                                # in place
        F.fvv_depth_jbf(rgb, 24, d, 16, d, 16, 8, 8, ok)
    assert e.value.code == F.FVV_ERR_INVALID_ARG
    with pytest.raises(F.FvvError) as e:                                # host memory
        F.fvv_depth_jbf(rgb, 24, np.zeros((8, 8), np.uint16), 16, o, 16, 8, 8, ok)
    assert e.value.code == F.FVV_ERR_INVALID_ARG
