"""Adaptive view transmission (Sec. V-C) on the GPU: ticks that carry only
the N_Tx cameras nearest the viewpoint.  A view renders from the newest
resident tick holding all of its active references and never reads the
other cameras' slots, so its result equals the oracle on the true frames
even where the other cameras' slots hold unrelated data."""
import numpy as np
import pytest

import synthetic as S
from fvv_helpers import assert_parity, lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def arc():
    return S.workload("plain_9cam_1280x720", scale=0.26)          # 333 x 187


def _render(F, ctx, v, ticks=None):
    import torch
    H, W = v.height, v.width
    keys = torch.zeros((H, W), dtype=torch.int64, device="cuda")
    kraw = torch.zeros((H, W), dtype=torch.int64, device="cuda")
    dep = torch.zeros((H, W), dtype=torch.float32, device="cuda")
    hole = torch.zeros((H, W), dtype=torch.uint8, device="cuda")
    top3 = torch.zeros((H, W, 3), dtype=torch.float32, device="cuda")
    out = torch.zeros((H, W * 3), dtype=torch.uint8, device="cuda")
    F.fvv_synthesize_batch(ctx, [v], ticks, [out], [W * 3], [F.aux(dep, hole, top3, keys, kraw)])
    torch.cuda.synchronize()
    return {"rgb": out.cpu().numpy().reshape(H, W, 3), "depth": dep.cpu().numpy(), "hole": hole.cpu().numpy(),
            "top3": top3.cpu().numpy(), "keys": keys.cpu().numpy().view(np.uint64),
            "keys_raw": kraw.cpu().numpy().view(np.uint64)}


def _packed(a, mask):
    return np.ascontiguousarray(np.stack([a[k] for k in range(len(a)) if (mask >> k) & 1]))


@pytest.mark.parametrize("device", [False, True])
def test_subset_tick_renders_like_the_full_frames(oracle_mod, arc, device):
    import torch
    F = lib()
    cams, rgb, dep = arc["cams"], arc["rgb"], arc["depth"]
    H, W = cams[0].height, cams[0].width
    rng = np.random.default_rng(9)
    junk_rgb = rng.integers(0, 256, rgb.shape).astype(np.uint8)
    junk_dep = rng.integers(300, 6000, dep.shape).astype(np.uint16)
    ctx = F.fvv_create(F.rig(cams, arc["look_at"]), F.fvv_default_options(n_ref=3, frame_slots=1))
    try:
        v = arc["views"][40]
        mask = F.fvv_select_cameras(F.rig(cams, arc["look_at"]), [v], 5)
        assert bin(mask).count("1") == 5
        # tick 0: every camera with unrelated frames; tick 1 (the same slot):
        # only the selected cameras, with the true frames
        F.fvv_upload_frames(ctx, junk_rgb, H * W * 3, W * 3, junk_dep, H * W * 2, W * 2, 0)
        r, d = _packed(rgb, mask), _packed(dep, mask)
        if device:
            r = torch.from_numpy(r).cuda()
            d = torch.from_numpy(d.view(np.int16)).cuda()
        F.fvv_upload_frames_subset(ctx, mask, r, H * W * 3, W * 3, d, H * W * 2, W * 2, 1)
        g = _render(F, ctx, v)
        ref = oracle_mod.synthesize(cams, rgb, dep, v, arc["look_at"], n_ref=3)
        assert_parity(g, ref, "subset tick")
        # a view whose references are not all in the tick cannot render
        rr = F.rig(cams, arc["look_at"])
        far = next(u for u in arc["views"] if F.fvv_select_cameras(rr, [u], 3) & ~mask)
        with pytest.raises(F.FvvError) as e:
            _render(F, ctx, far)
        assert e.value.code == F.FVV_ERR_NOT_READY
        with pytest.raises(F.FvvError) as e:
            _render(F, ctx, far, ticks=[1])
        assert e.value.code == F.FVV_ERR_NOT_READY
    finally:
        F.fvv_destroy(ctx)


def test_view_uses_the_newest_tick_holding_its_cameras(oracle_mod, arc):
    """Tick 5 carries every camera (frames A), tick 6 only some (frames B):
    a view whose references tick 6 holds renders B, another renders A."""
    F = lib()
    cams, rgb, dep = arc["cams"], arc["rgb"], arc["depth"]
    H, W = cams[0].height, cams[0].width
    rgb_b = np.ascontiguousarray(rgb[:, :, :, ::-1])
    r = F.rig(cams, arc["look_at"])
    ctx = F.fvv_create(r, F.fvv_default_options(n_ref=3, frame_slots=4))
    try:
        va, vb = arc["views"][225], arc["views"][75]               # phi = -22.5 and +22.5 deg
        mb = F.fvv_select_cameras(r, [vb], 3)
        ma = F.fvv_select_cameras(r, [va], 3)
        assert ma & ~mb
        F.fvv_upload_frames(ctx, rgb, H * W * 3, W * 3, dep, H * W * 2, W * 2, 5)
        F.fvv_upload_frames_subset(ctx, mb, _packed(rgb_b, mb), H * W * 3, W * 3, _packed(dep, mb),
                                   H * W * 2, W * 2, 6)
        assert F.fvv_latest_tick(ctx) == 5                      # the newest tick holding every camera
        gb = _render(F, ctx, vb)
        assert_parity(gb, oracle_mod.synthesize(cams, rgb_b, dep, vb, arc["look_at"], n_ref=3), "tick 6")
        ga = _render(F, ctx, va)
        assert_parity(ga, oracle_mod.synthesize(cams, rgb, dep, va, arc["look_at"], n_ref=3), "tick 5")
        with pytest.raises(F.FvvError) as e:
            F.fvv_upload_frames_subset(ctx, 0, rgb, H * W * 3, W * 3, dep, H * W * 2, W * 2, 7)
        assert e.value.code == F.FVV_ERR_INVALID_ARG
        with pytest.raises(F.FvvError) as e:
            F.fvv_upload_frames_subset(ctx, 1 << 9, rgb, H * W * 3, W * 3, dep, H * W * 2, W * 2, 7)
        assert e.value.code == F.FVV_ERR_INVALID_ARG
    finally:
        F.fvv_destroy(ctx)
