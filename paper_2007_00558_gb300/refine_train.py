"""Leave-one-camera-out (LOO) training of the refinement network.

For every camera j of a rig, the plain method synthesises camera j's own
viewpoint from the other cameras; the camera's real frame is the target.
These pairs train the U-Net (fvv_refine_train_step) and measure what it gains
over the plain synthesis.  All synthesis and training runs in the library's
kernels; torch only holds device tensors and assembles batches.
"""
from __future__ import annotations

import math
from typing import List, Sequence

import numpy as np

from . import fvv as F


class LooRig:
    """One context per held-out camera j, over the rig without camera j."""

    def __init__(self, cams: Sequence, look_at, opts=None):
        self.cams = list(cams)
        self.ctxs = []
        for j in range(len(self.cams)):
            others = [c for i, c in enumerate(self.cams) if i != j]
            self.ctxs.append(F.fvv_create(F.rig(others, look_at), opts))
        self.tick = 0

    def close(self):
        for c in self.ctxs:
            F.fvv_destroy(c)
        self.ctxs = []

    def samples(self, rgb: np.ndarray, depth: np.ndarray, target_rgb: np.ndarray = None) -> dict:
        """LOO samples of one set of frames (K, H, W, 3) / (K, H, W).
        Returns device tensors rgb, depth, hole, top3, target: (K, H, W, ...)."""
        import torch
        K, H, W = depth.shape
        target_rgb = rgb if target_rgb is None else target_rgb
        out = {"rgb": torch.empty((K, H, W, 3), dtype=torch.uint8, device="cuda"),
               "depth": torch.empty((K, H, W), dtype=torch.float32, device="cuda"),
               "hole": torch.empty((K, H, W), dtype=torch.uint8, device="cuda"),
               "top3": torch.empty((K, H, W, 3), dtype=torch.float32, device="cuda")}
        t = self.tick
        self.tick += 1
        for j, ctx in enumerate(self.ctxs):
            k = 0
            for i in range(K):
                if i == j:
                    continue
                F.fvv_upload_frame(ctx, k, np.ascontiguousarray(rgb[i]), W * 3,
                                   np.ascontiguousarray(depth[i]), W * 2, t)
                k += 1
            aux = F.aux(depth=out["depth"][j], hole=out["hole"][j], top3=out["top3"][j])
            F.fvv_synthesize(ctx, self.cams[j], out["rgb"][j], W * 3, aux)
        torch.cuda.synchronize()
        out["target"] = torch.from_numpy(np.ascontiguousarray(target_rgb)).cuda()
        return out


def concat(samples: List[dict]) -> dict:
    import torch
    return {k: torch.cat([s[k] for s in samples], 0).contiguous() for k in samples[0]}


def _crop(data: dict, idx, y0, x0, h, w) -> dict:
    return {k: v[idx, y0:y0 + h, x0:x0 + w].contiguous() for k, v in data.items()}


def train(ctx: int, data: dict, steps: int, batch: int = 8, crop: int = 128, lr: float = 2e-3,
          seed: int = 0, lr_final: float = 2e-4) -> List[float]:
    """Adam on random crops of random LOO samples (cosine learning-rate decay)."""
    import torch
    n, H, W = data["depth"].shape
    rng = np.random.default_rng(seed)
    ch, cw = min(crop, H) // 4 * 4, min(crop, W) // 4 * 4
    losses = []
    for s in range(steps):
        idx = torch.from_numpy(rng.integers(0, n, batch)).cuda()
        y0 = int(rng.integers(0, H - ch + 1))
        x0 = int(rng.integers(0, W - cw + 1))
        b = _crop(data, idx, y0, x0, ch, cw)
        rate = lr_final + 0.5 * (lr - lr_final) * (1 + math.cos(math.pi * s / max(1, steps - 1)))
        fb = F.refine_batch(batch, ch, cw, b["rgb"], b["depth"], b["hole"], b["top3"], b["target"])
        losses.append(F.fvv_refine_train_step(ctx, fb, rate))
    return losses


def quantize(ctx: int, data: dict, n: int = 8) -> None:
    """E4M3 inference for `ctx`: activation scales from a bf16 pass over the
    first n samples of `data` (full frames, cropped to multiples of 4)."""
    _, H, W = data["depth"].shape
    h4, w4 = H // 4 * 4, W // 4 * 4
    n = min(n, data["depth"].shape[0])
    b = {k: v[:n, :h4, :w4].contiguous() for k, v in data.items()}
    fb = F.refine_batch(n, h4, w4, b["rgb"], b["depth"], b["hole"], b["top3"])
    F.fvv_refine_quantize(ctx, fb)


def psnr(a, b) -> float:
    d = (a.float() - b.float())
    mse = float((d * d).mean())
    return float("inf") if mse == 0 else 10 * math.log10(255.0 ** 2 / mse)


def evaluate(ctx: int, data: dict, chunk: int = 8) -> dict:
    """PSNR of the plain synthesis and of the refined one against the
    held-out cameras, over all samples (full frames, cropped to multiples of 4)."""
    import torch
    n, H, W = data["depth"].shape
    h4, w4 = H // 4 * 4, W // 4 * 4
    refined = torch.empty((n, h4, w4, 3), dtype=torch.uint8, device="cuda")
    for i in range(0, n, chunk):
        j = min(n, i + chunk)
        b = {k: v[i:j, :h4, :w4].contiguous() for k, v in data.items()}
        fb = F.refine_batch(j - i, h4, w4, b["rgb"], b["depth"], b["hole"], b["top3"])
        F.fvv_refine_forward(ctx, fb, refined[i:j])
    tgt = data["target"][:, :h4, :w4]
    plain = data["rgb"][:, :h4, :w4]
    hole = data["hole"][:, :h4, :w4].bool()
    return {"psnr_plain": psnr(plain, tgt), "psnr_refined": psnr(refined, tgt),
            "psnr_plain_holes": psnr(plain[hole], tgt[hole]) if bool(hole.any()) else None,
            "psnr_refined_holes": psnr(refined[hole], tgt[hole]) if bool(hole.any()) else None,
            "samples": n, "size": "%dx%d" % (w4, h4)}
