"""GPU parity of layered FG/BG synthesis (Sec. VI: per-camera FG and BG
layers, mixed separately and stacked) against oracle.synthesize_layered on
the same seeded inputs: the keys of the layer shown, the FG layer's raw
keys, hole mask and depth bit-exact; colour within 1/255 on >= 99.9 % of
pixels (fvv_helpers.assert_parity)."""
import numpy as np
import pytest

import synthetic as S
from oracle import codec as K
from fvv_helpers import assert_parity, gpu_run, lib

pytestmark = pytest.mark.gpu


def _opts(**kw):
    return lib().fvv_default_options(layered=1, **kw)


@pytest.fixture(scope="module")
def lay_small():
    return S.workload("layered_9cam_1280x720", scale=0.26)     # 333 x 187: ragged rows


@pytest.fixture(scope="module")
def lay_full():
    return S.workload("layered_9cam_1280x720")


def _check(oracle_mod, wl, views, bg="model", **kw):
    models = wl["bg"] if bg == "model" else None
    gs = gpu_run(wl["cams"], wl["rgb"], wl["depth"], views, wl["look_at"], opts=_opts(**kw), bg=models)
    out = []
    for i, (g, v) in enumerate(zip(gs, views)):
        ref = oracle_mod.synthesize_layered(wl["cams"], wl["rgb"], wl["depth"], models, v, wl["look_at"], **kw)
        out.append(assert_parity(g, ref, "view %d %s" % (i, kw)))
        assert (ref["layer"] == 0).any()
        if models is not None:
            assert (ref["layer"] == 1).any()
    return out


def test_layered_small_batch(oracle_mod, lay_small):
    wl = lay_small
    _check(oracle_mod, wl, [wl["views"][i] for i in (0, 75, 210)])


@pytest.mark.parametrize("kw", [dict(crack_filter=0), dict(hole_fill=0), dict(n_ref=3),
                                dict(crack_filter=0, hole_fill=0, n_ref=2), dict(pixel_weights=1)])
def test_layered_options(oracle_mod, lay_small, kw):
    wl = lay_small
    _check(oracle_mod, wl, [wl["views"][40]], **kw)


def test_layered_without_models(oracle_mod, lay_small):
    """Layered with no background model: BG-signalled pixels are not warped."""
    wl = lay_small
    _check(oracle_mod, wl, [wl["views"][120]], bg=None)


def test_layered_full_size(oracle_mod, lay_full):
    wl = lay_full
    for info in _check(oracle_mod, wl, [wl["views"][i] for i in (37, 150)]):
        assert info["exact_rgb_fraction"] >= 0.999


def test_single_layer_treats_the_background_signal_as_no_depth(oracle_mod, lay_small):
    """Without layered, BG-signalled pixels are outside [d_lo, d_hi]: the
    single-layer oracle on the same frames is the reference."""
    wl = lay_small
    v = wl["views"][60]
    g = gpu_run(wl["cams"], wl["rgb"], wl["depth"], [v], wl["look_at"], bg=wl["bg"])[0]
    ref = oracle_mod.synthesize(wl["cams"], wl["rgb"], wl["depth"], v, wl["look_at"])
    assert_parity(g, ref, "single layer")
    assert ref["hole"].mean() > 0.3


def test_layered_from_yuv420_depth(oracle_mod, lay_small):
    """The transmission chain: live depth with background pixels encoded to
    YUV420 (Eq. (1)-(3), code 0 for BG), uploaded through the fused decode,
    then layered synthesis; against the oracle on the oracle-decoded depth."""
    import torch
    F = lib()
    wl = lay_small
    cams = wl["cams"]
    H, W = cams[0].height, cams[0].width
    H2, W2 = H - H % 2, W - W % 2                       # the codec needs even sizes
    cams2 = [c.copy() for c in cams]
    for c in cams2:
        c.width, c.height = W2, H2
    rgb = np.ascontiguousarray(wl["rgb"][:, :H2, :W2])
    live = np.ascontiguousarray(wl["depth"][:, :H2, :W2])
    model = np.ascontiguousarray(wl["bg"][:, :H2, :W2])
    codec = dict(z_near=0.3, z_far=8.0, alpha=0.0, beta=1.0)
    ctx = F.fvv_create(F.rig(cams2, wl["look_at"]), _opts())
    try:
        dec = []
        for k in range(len(cams2)):
            F.fvv_set_depth_codec(ctx, k, F.fvv_depth_codec_default(**codec))
            F.fvv_set_bg_depth(ctx, k, model[k], W2 * 2)
            y, u, v = K.encode(live[k], unit_m=0.001, **codec)
            dec.append(K.decode(y, u, v, codec["z_near"], codec["z_far"], 0.001))
            F.fvv_upload_frame_yuv(ctx, k, rgb[k], W2 * 3, y, W2, u, v, W2 // 2, 0)
        dec = np.stack(dec)
        assert (dec == S.DEPTH_BG).mean() > 0.3
        view = wl["views"][90].copy()
        view.width, view.height = W2, H2
        keys = torch.zeros((H2, W2), dtype=torch.int64, device="cuda")
        out = torch.zeros((H2, W2 * 3), dtype=torch.uint8, device="cuda")
        F.fvv_synthesize(ctx, view, out, W2 * 3, F.aux(keys=keys))
        torch.cuda.synchronize()
        ref = oracle_mod.synthesize_layered(cams2, rgb, dec, model, view, wl["look_at"])
        assert np.array_equal(keys.cpu().numpy().view(np.uint64), ref["keys"])
        d = np.abs(out.cpu().numpy().reshape(H2, W2, 3).astype(int) - ref["rgb"].astype(int))
        assert (d <= 1).all(axis=-1).mean() >= 0.999
    finally:
        F.fvv_destroy(ctx)


def test_bg_model_errors():
    F = lib()
    cams = S.rig_arc(2, 30.0, 1.5, 40, 30, 40.0)
    ctx = F.fvv_create(F.rig(cams, [0, 0, 0]), _opts())
    try:
        m = np.full((30, 40), 1500, np.uint16)
        for cam, pitch in ((2, 80), (-1, 80), (0, 78), (0, 81)):
            with pytest.raises(F.FvvError) as e:
                F.fvv_set_bg_depth(ctx, cam, m, pitch)
            assert e.value.code == F.FVV_ERR_INVALID_ARG
        F.fvv_set_bg_depth(ctx, 0, m, 80)
        F.fvv_set_bg_depth(ctx, 0, None)                  # removed again
    finally:
        F.fvv_destroy(ctx)
