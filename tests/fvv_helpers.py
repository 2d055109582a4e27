"""Helpers for the tests: run the CUDA path through the C ABI, compare with
the oracle."""
import math

import numpy as np

KEY_EMPTY = np.uint64(0xFFFFFFFFFFFFFFFF)


def lib():
    from paper_2007_00558_gb300 import build, fvv
    build.build()
    fvv.load()
    return fvv


def gpu_run(cams, rgb, depth, views, look_at, opts=None, ticks=None, host_out=False,
            rgb_pitch_pad=0, depth_pitch_pad=0, out_pitch_pad=0, stream=None, bg=None):
    """Upload one tick (0) of frames (and, with ``bg``, each camera's
    background depth model) and synthesise ``views`` in one batch.

    Returns a list of dicts (rgb, depth, hole, top3, keys, keys_raw) as numpy.
    """
    import torch
    F = lib()
    r = F.rig(cams, look_at)
    ctx = F.fvv_create(r, opts)
    try:
        for k, c in enumerate(cams):
            if bg is not None and bg[k] is not None:
                F.fvv_set_bg_depth(ctx, k, np.ascontiguousarray(bg[k], np.uint16), c.width * 2)
        for k, c in enumerate(cams):
            H, W = c.height, c.width
            rp = W * 3 + rgb_pitch_pad
            dp = W * 2 + depth_pitch_pad
            rbuf = np.zeros((H, rp), np.uint8)
            rbuf[:, :W * 3] = np.asarray(rgb[k]).reshape(H, W * 3)
            dbuf = np.zeros((H, dp // 2 + (dp % 2)), np.uint16).view(np.uint8)[:, :dp].copy()
            dbuf[:, :W * 2] = np.asarray(depth[k], np.uint16).view(np.uint8).reshape(H, W * 2)
            F.fvv_upload_frame(ctx, k, rbuf, rp, dbuf, dp, 0, stream)
        outs, pitches, auxs, res = [], [], [], []
        for v in views:
            H, W = v.height, v.width
            op = W * 3 + out_pitch_pad
            if host_out:
                o = {"rgb_buf": np.zeros((H, op), np.uint8),
                     "depth": np.zeros((H, W), np.float32), "hole": np.zeros((H, W), np.uint8),
                     "top3": np.zeros((H, W, 3), np.float32), "keys": np.zeros((H, W), np.uint64),
                     "keys_raw": np.zeros((H, W), np.uint64)}
            else:
                dev = torch.device("cuda")
                o = {"rgb_buf": torch.zeros((H, op), dtype=torch.uint8, device=dev),
                     "depth": torch.zeros((H, W), dtype=torch.float32, device=dev),
                     "hole": torch.zeros((H, W), dtype=torch.uint8, device=dev),
                     "top3": torch.zeros((H, W, 3), dtype=torch.float32, device=dev),
                     "keys": torch.zeros((H, W), dtype=torch.int64, device=dev),
                     "keys_raw": torch.zeros((H, W), dtype=torch.int64, device=dev)}
            outs.append(o["rgb_buf"])
            pitches.append(op)
            auxs.append(F.aux(o["depth"], o["hole"], o["top3"], o["keys"], o["keys_raw"]))
            res.append(o)
        F.fvv_synthesize_batch(ctx, views, ticks, outs, pitches, auxs, stream)
        torch.cuda.synchronize()
    finally:
        F.fvv_destroy(ctx)
    out = []
    for v, o in zip(views, res):
        H, W = v.height, v.width
        g = {k: (x.cpu().numpy() if hasattr(x, "cpu") else x) for k, x in o.items()}
        g["rgb"] = g.pop("rgb_buf")[:, :W * 3].reshape(H, W, 3)
        g["keys"] = g["keys"].view(np.uint64)
        g["keys_raw"] = g["keys_raw"].view(np.uint64)
        out.append(g)
    return out


def psnr(a, b):
    mse = np.mean((np.asarray(a, float) - np.asarray(b, float)) ** 2)
    return float("inf") if mse == 0 else 10 * math.log10(255.0 ** 2 / mse)


def assert_parity(gpu, ref, label=""):
    """The parity bar: z-buffer keys (before and after the filter), hole mask
    and depth bit-exact; colour within 1/255 per channel on >= 99.9 % of
    pixels with PSNR >= 50 dB; top-3 weights within 1e-6 relative."""
    assert np.array_equal(gpu["keys_raw"], ref["keys_raw"]), label + ": raw keys differ at %d px" % \
        int((gpu["keys_raw"] != ref["keys_raw"]).sum())
    assert np.array_equal(gpu["keys"], ref["keys"]), label + ": filtered keys differ"
    assert np.array_equal(gpu["hole"], ref["hole"]), label + ": hole mask differs"
    assert np.array_equal(gpu["depth"], ref["depth"]), label + ": depth differs"
    d = np.abs(gpu["rgb"].astype(int) - ref["rgb"].astype(int))
    within = (d <= 1).all(axis=-1).mean()
    assert within >= 0.999, label + ": only %.5f of pixels within 1/255" % within
    assert psnr(gpu["rgb"], ref["rgb"]) >= 50.0, label + ": PSNR %.2f" % psnr(gpu["rgb"], ref["rgb"])
    assert np.allclose(gpu["top3"], ref["top3"], rtol=1e-6, atol=0), label + ": top3 differ"
    return {"exact_rgb_fraction": float((d == 0).all(axis=-1).mean())}
