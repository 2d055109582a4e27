"""The refinement network at the size it is timed at (a batch of four
1280x720 views, the launch configuration of the refine throughput run)
against the FP64 oracle (oracle/unet.py) on sampled windows.

The oracle cannot run the whole batch, but an output pixel depends only on
the inputs within its receptive field (about 24 pixels here: two 3x3 layers
at each of the three scales on the way down and up).  So each sample runs
the oracle on a 128 x 128 crop whose origin is a multiple of 4 (the pooling
grids of crop and image coincide) and compares the pixels at least 40 pixels
from every crop edge that is not an image edge (where both sides pad with
zeros).  The crops cover the image corners, where the tiles are ragged, and
the interior.  Bound: the residual within 3 % relative L2 of the oracle's,
as for the small-size test (bf16 activations, fp32 accumulation)."""
import numpy as np
import pytest

from oracle import unet as U
from fvv_helpers import lib

pytestmark = pytest.mark.gpu

Z_FAR = 8000.0
S, MARGIN = 128, 40


def _bf16_round(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(torch.bfloat16).double().numpy()


def _flat(p):
    parts = []
    for name in U.LAYERS_3x3:
        parts += [p[name + ".w"].reshape(-1), p[name + ".b"]]
    parts += [p["out.w"].reshape(-1), p["out.b"]]
    return np.concatenate(parts)


@pytest.mark.parametrize("widths", [(32, 64, 128), (48, 96, 192)])
def test_full_size_batch_matches_oracle_on_windows(widths):
    import torch
    F = lib()
    import synthetic as Syn
    cams = Syn.rig_parallel(1, 16, 16, 10.0, 0.1)
    ctx = F.fvv_create(F.rig(cams, [0, 0, 1]))
    try:
        F.fvv_refine_init(ctx, F.fvv_refine_default_cfg(widths=widths, z_far=Z_FAR))
        rng = np.random.default_rng(sum(widths))
        p = U.init_params(widths, seed=5, out_scale=0.3)
        for k in p:
            if k.endswith(".b"):
                p[k] = rng.standard_normal(p[k].shape) * 0.05
        F.fvv_refine_set(ctx, F.FVV_REFINE_PARAMS, _flat(p))
        n, H, W = 4, 720, 1280
        rgb = rng.integers(40, 216, (n, H, W, 3)).astype(np.uint8)
        depth = rng.uniform(800, 6000, (n, H, W)).astype(np.float32)
        hole = (rng.random((n, H, W)) < 0.1).astype(np.uint8)
        top3 = rng.dirichlet([2, 1, 1], (n, H, W)).astype(np.float32)
        dev = [torch.from_numpy(a).cuda() for a in (rgb, depth, hole, top3)]
        b = F.refine_batch(n, H, W, *dev, None)
        out = torch.zeros((n, H, W, 3), dtype=torch.float32, device="cuda")
        F.fvv_refine_forward(ctx, b, None, out)
        got = out.double().cpu().numpy()
    finally:
        F.fvv_destroy(ctx)
    pw = {k: _bf16_round(v) if k.endswith(".w") and not k.startswith("out") else v for k, v in p.items()}
    # (image, crop origin y, x): the four corners and two interior windows
    crops = [(0, 0, 0), (1, 0, W - S), (2, H - S, 0), (3, H - S, W - S), (0, 296, 604), (2, 400, 1000)]
    for i, y0, x0 in crops:
        sl = (slice(i, i + 1), slice(y0, y0 + S), slice(x0, x0 + S))
        feat = U.features(rgb[sl], depth[sl], hole[sl], top3[sl], Z_FAR)
        c_rgb = rgb[sl].astype(np.float64) / 255.0
        pred, _ = U.forward(pw, _bf16_round(feat), c_rgb)
        t = 0 if y0 == 0 else MARGIN
        bt = S if y0 + S == H else S - MARGIN
        l = 0 if x0 == 0 else MARGIN
        r = S if x0 + S == W else S - MARGIN
        res_ref = pred[0, t:bt, l:r] - c_rgb[0, t:bt, l:r]
        res_gpu = got[i, y0 + t:y0 + bt, x0 + l:x0 + r] - c_rgb[0, t:bt, l:r]
        rel = np.linalg.norm(res_gpu - res_ref) / np.linalg.norm(res_ref)
        assert rel <= 0.03, (widths, i, y0, x0, rel)


@pytest.mark.parametrize("widths", [(32, 64, 128), (48, 96, 192)])
def test_full_size_e4m3_batch_matches_quantised_oracle_on_windows(widths):
    """The E4M3 form on the full-size batch, against the oracle's quantised
    forward pass (forward_e4m3) on the same windows with the same activation
    scales.  As in the small-size E4M3 test, a value within fp32 noise of an
    E4M3 tie may land on either neighbour, so the bound is 3x the oracle's own
    spread when its scales move by 1e-6 (at least 1 %); the 8-bit output is the
    rounded float output everywhere."""
    import torch
    F = lib()
    import synthetic as Syn
    cams = Syn.rig_parallel(1, 16, 16, 10.0, 0.1)
    ctx = F.fvv_create(F.rig(cams, [0, 0, 1]))
    try:
        F.fvv_refine_init(ctx, F.fvv_refine_default_cfg(widths=widths, z_far=Z_FAR))
        rng = np.random.default_rng(7 + sum(widths))
        p = U.init_params(widths, seed=8, out_scale=0.5)
        for k in p:
            if k.endswith(".b"):
                p[k] = rng.standard_normal(p[k].shape) * 0.05
        F.fvv_refine_set(ctx, F.FVV_REFINE_PARAMS, _flat(p))
        p32 = {k: v.astype(np.float32).astype(np.float64) for k, v in p.items()}
        n, H, W = 4, 720, 1280
        rgb = rng.integers(40, 216, (n, H, W, 3)).astype(np.uint8)
        depth = rng.uniform(800, 6000, (n, H, W)).astype(np.float32)
        hole = (rng.random((n, H, W)) < 0.1).astype(np.uint8)
        top3 = rng.dirichlet([2, 1, 1], (n, H, W)).astype(np.float32)
        # activation scales from the oracle's FP64 pass over one window
        sl0 = (slice(0, 1), slice(296, 296 + S), slice(604, 604 + S))
        x0 = U.features(rgb[sl0], depth[sl0], hole[sl0], top3[sl0], Z_FAR)
        _, cache = U.forward(p32, x0, rgb[sl0].astype(np.float64) / 255.0)
        scales = U.activation_scales(cache)
        F.fvv_refine_quantize(ctx, None, scales.astype(np.float32))
        dev = [torch.from_numpy(a).cuda() for a in (rgb, depth, hole, top3)]
        b = F.refine_batch(n, H, W, *dev, None)
        out = torch.zeros((n, H, W, 3), dtype=torch.float32, device="cuda")
        out8 = torch.zeros((n, H, W, 3), dtype=torch.uint8, device="cuda")
        F.fvv_refine_forward(ctx, b, out8, out)
        got = out.double().cpu().numpy()
        assert np.array_equal(out8.cpu().numpy(), np.floor(out.cpu().numpy() * 255.0 + 0.5).astype(np.uint8))
    finally:
        F.fvv_destroy(ctx)
    s32 = scales.astype(np.float32).astype(np.float64)
    for i, y0, x0 in [(0, 0, 0), (3, H - S, W - S), (1, 296, 604), (2, 0, W - S)]:
        sl = (slice(i, i + 1), slice(y0, y0 + S), slice(x0, x0 + S))
        x = U.features(rgb[sl], depth[sl], hole[sl], top3[sl], Z_FAR)
        c_rgb = rgb[sl].astype(np.float64) / 255.0
        t = 0 if y0 == 0 else MARGIN
        bt = S if y0 + S == H else S - MARGIN
        l = 0 if x0 == 0 else MARGIN
        r = S if x0 + S == W else S - MARGIN

        def win(a):
            return a[0, t:bt, l:r] - c_rgb[0, t:bt, l:r]

        def rel(a, b):
            return np.linalg.norm(win(a) - win(b)) / np.linalg.norm(win(b))
        ref = U.forward_e4m3(p32, x, c_rgb, s32)
        spread = max(rel(U.forward_e4m3(p32, x, c_rgb, s32 * (1 + 1e-6)), ref),
                     rel(U.forward_e4m3(p32, x, c_rgb, s32 * (1 - 1e-6)), ref), 0.01)
        g = got[i:i + 1, y0:y0 + S, x0:x0 + S]
        assert rel(g, ref) <= 3.0 * spread, (widths, i, y0, x0, rel(g, ref), spread)
