"""The refinement network on the GPU against the FP64 oracle (oracle/unet.py).

Same weights (copied into the GPU net) and the same bf16-rounded input
features.  The GPU keeps activations in bf16 and accumulates in fp32, so the
bound is stated per quantity: forward residual within 3 % relative L2 of the
oracle's; every layer's weight gradient within 5 % relative L2 and cosine
similarity >= 0.998."""
import os
import tempfile

import numpy as np
import pytest

from oracle import unet as U
import synthetic as S
from fvv_helpers import lib

pytestmark = pytest.mark.gpu

WIDTHS = (32, 64, 128)
Z_FAR = 8000.0


def _bf16_round(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(torch.bfloat16).double().numpy()


def _flat(p):
    parts = []
    for name in U.LAYERS_3x3:
        parts += [p[name + ".w"].reshape(-1), p[name + ".b"]]
    parts += [p["out.w"].reshape(-1), p["out.b"]]
    return np.concatenate(parts)


def _unflat(v, widths=WIDTHS):
    shapes = U.layer_shapes(widths)
    out, o = {}, 0
    for name in U.LAYERS_3x3 + ["out"]:
        co, ci = shapes[name]
        n = co * ci * (9 if name != "out" else 1)
        out[name + ".w"] = v[o:o + n].reshape((co, 3, 3, ci) if name != "out" else (co, ci))
        o += n
        out[name + ".b"] = v[o:o + co]
        o += co
    assert o == v.size
    return out


def _batch(rng, n, h, w):
    import torch
    rgb = rng.integers(60, 196, (n, h, w, 3)).astype(np.uint8)
    depth = rng.uniform(800, 6000, (n, h, w)).astype(np.float32)
    hole = (rng.random((n, h, w)) < 0.1).astype(np.uint8)
    top3 = rng.dirichlet([2, 1, 1], (n, h, w)).astype(np.float32)
    target = np.clip(rgb.astype(int) + rng.integers(-30, 31, rgb.shape), 0, 255).astype(np.uint8)
    dev = {k: torch.from_numpy(v).cuda() for k, v in
           dict(rgb=rgb, depth=depth, hole=hole, top3=top3, target=target).items()}
    host = dict(rgb=rgb, depth=depth, hole=hole, top3=top3, target=target)
    return host, dev


def _oracle_inputs(h):
    feat = U.features(h["rgb"], h["depth"], h["hole"], h["top3"], Z_FAR)
    return _bf16_round(feat), h["rgb"].astype(np.float64) / 255.0, h["target"].astype(np.float64) / 255.0


@pytest.fixture()
def net():
    F = lib()
    cams = S.rig_parallel(1, 16, 16, 10.0, 0.1)
    ctx = F.fvv_create(F.rig(cams, [0, 0, 1]))
    F.fvv_refine_init(ctx, F.fvv_refine_default_cfg(widths=WIDTHS, z_far=Z_FAR))
    yield F, ctx
    F.fvv_destroy(ctx)


def test_forward_and_gradients_match_oracle(net):
    import torch
    F, ctx = net
    rng = np.random.default_rng(0)
    p = U.init_params(WIDTHS, seed=3, out_scale=0.3)
    for k in p:
        if k.endswith(".b"):
            p[k] = rng.standard_normal(p[k].shape) * 0.05
    F.fvv_refine_set(ctx, F.FVV_REFINE_PARAMS, _flat(p))
    n, h, w = 2, 32, 48
    host, dev = _batch(rng, n, h, w)
    b = F.refine_batch(n, h, w, dev["rgb"], dev["depth"], dev["hole"], dev["top3"], dev["target"])
    out = torch.zeros((n, h, w, 3), dtype=torch.float32, device="cuda")
    F.fvv_refine_forward(ctx, b, None, out)
    x, rgb, target = _oracle_inputs(host)
    pw = {k: _bf16_round(v) if k.endswith(".w") and not k.startswith("out") else v for k, v in p.items()}
    pred, cache = U.forward(pw, x, rgb)
    res_gpu = out.double().cpu().numpy() - np.clip(rgb, 0, 1)
    res_ref = pred - np.clip(rgb, 0, 1)
    rel = np.linalg.norm(res_gpu - res_ref) / np.linalg.norm(res_ref)
    assert rel <= 0.03, rel
    # gradients (lr = 0: forward + backward, no update)
    loss_gpu = F.fvv_refine_train_step(ctx, b, 0.0)
    loss_ref, dpred = U.mse(pred, target)
    assert abs(loss_gpu - loss_ref) <= 0.02 * loss_ref
    g_ref = U.backward(pw, cache, dpred)
    g_gpu = _unflat(F.fvv_refine_get(ctx, F.FVV_REFINE_GRADS).astype(np.float64))
    for k in g_ref:
        a, r = g_gpu[k].reshape(-1), g_ref[k].reshape(-1)
        rel = np.linalg.norm(a - r) / max(np.linalg.norm(r), 1e-12)
        cos = a @ r / max(np.linalg.norm(a) * np.linalg.norm(r), 1e-30)
        assert rel <= 0.05 and cos >= 0.998, (k, rel, cos)
    # nothing was updated
    assert np.array_equal(F.fvv_refine_get(ctx, F.FVV_REFINE_PARAMS), _flat(p).astype(np.float32))
    # every reduction has a fixed order: the same step gives the same bits
    g1 = F.fvv_refine_get(ctx, F.FVV_REFINE_GRADS)
    assert F.fvv_refine_train_step(ctx, b, 0.0) == loss_gpu
    assert np.array_equal(F.fvv_refine_get(ctx, F.FVV_REFINE_GRADS), g1)


def test_training_reduces_loss_and_checkpoint_round_trip(net):
    import torch
    F, ctx = net
    rng = np.random.default_rng(1)
    n, h, w = 4, 64, 64
    host, dev = _batch(rng, n, h, w)
    # a learnable target: the inverted colour (a linear function of the input)
    dev["target"] = (255 - dev["rgb"]).contiguous()
    b = F.refine_batch(n, h, w, dev["rgb"], dev["depth"], dev["hole"], dev["top3"], dev["target"])
    losses = [F.fvv_refine_train_step(ctx, b, 2e-3) for _ in range(160)]
    print("training losses", losses[0], losses[40], losses[80], losses[-1])
    assert losses[-1] < 0.25 * losses[0], (losses[0], losses[-1])
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "unet.bin")
        F.fvv_refine_save(ctx, path)
        cams = S.rig_parallel(1, 16, 16, 10.0, 0.1)
        ctx2 = F.fvv_create(F.rig(cams, [0, 0, 1]))
        try:
            F.fvv_refine_load(ctx2, path)
            for which in (F.FVV_REFINE_PARAMS, F.FVV_REFINE_ADAM_M, F.FVV_REFINE_ADAM_V):
                assert np.array_equal(F.fvv_refine_get(ctx, which), F.fvv_refine_get(ctx2, which))
            o1 = torch.zeros((n, h, w, 3), dtype=torch.uint8, device="cuda")
            o2 = torch.zeros_like(o1)
            F.fvv_refine_forward(ctx, b, o1)
            F.fvv_refine_forward(ctx2, b, o2)
            assert torch.equal(o1, o2)
            # every gradient is reduced in a fixed order: the resumed run
            # follows the original bit for bit
            for _ in range(3):
                l1 = F.fvv_refine_train_step(ctx, b, 2e-3)
                l2 = F.fvv_refine_train_step(ctx2, b, 2e-3)
                assert l1 == l2
            for which in (F.FVV_REFINE_PARAMS, F.FVV_REFINE_ADAM_M, F.FVV_REFINE_ADAM_V):
                assert np.array_equal(F.fvv_refine_get(ctx, which), F.fvv_refine_get(ctx2, which))
        finally:
            F.fvv_destroy(ctx2)


def test_synthesize_refined_runs_and_starts_near_plain():
    import torch
    F = lib()
    wl = S.workload("plain_9cam_1280x720", scale=0.25)        # 320 x 180
    ctx = F.fvv_create(F.rig(wl["cams"], wl["look_at"]))
    try:
        H, W = wl["cams"][0].height, wl["cams"][0].width
        for k in range(9):
            F.fvv_upload_frame(ctx, k, np.ascontiguousarray(wl["rgb"][k]), W * 3,
                               np.ascontiguousarray(wl["depth"][k]), W * 2, 0)
        F.fvv_refine_init(ctx, F.fvv_refine_default_cfg(seed=5))
        v = wl["views"][40]
        plain = torch.zeros((H, W * 3), dtype=torch.uint8, device="cuda")
        ref = torch.zeros_like(plain)
        F.fvv_synthesize(ctx, v, plain, W * 3)
        F.fvv_synthesize_refined(ctx, v, ref, W * 3)
        host = np.zeros((H, W * 3), np.uint8)
        F.fvv_synthesize_refined(ctx, v, host, W * 3)
        torch.cuda.synchronize()
        a, b = plain.cpu().numpy().astype(int), ref.cpu().numpy().astype(int)
        assert np.array_equal(host, ref.cpu().numpy())
        # an untrained head adds a small residual only
        assert np.abs(a - b).mean() < 20
    finally:
        F.fvv_destroy(ctx)
