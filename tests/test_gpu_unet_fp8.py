"""FP8 (E4M3) inference form of the refinement network on the GPU.

Against the oracle's quantised forward pass (oracle/unet.py forward_e4m3)
with the same activation scales -- the oracle's own, from its FP64 forward
pass -- and the same fp32 weights: both sides round every activation and
weight to E4M3 the same way.  Each E4M3 convolution alone matches the
oracle to one E4M3 step (test_gpu_unet_conv.py).  Through ten quantised
layers, though, a value within fp32 noise of an E4M3 tie lands on either
neighbour and the flip propagates: the oracle itself moves by several
percent when its scales move by 1e-6.  So the whole-network bounds are
stated against that measured sensitivity: the GPU stays within 3x the
oracle's tie-flip spread of the oracle, and its quantisation error (against
the FP64 network) equals the oracle's within 25 %."""
import numpy as np
import pytest

from oracle import unet as U
from fvv_helpers import lib
from test_gpu_unet_net import _batch, _flat, _oracle_inputs

pytestmark = pytest.mark.gpu

Z_FAR = 8000.0


def _net(F, widths):
    import synthetic as S
    cams = S.rig_parallel(1, 16, 16, 10.0, 0.1)
    ctx = F.fvv_create(F.rig(cams, [0, 0, 1]))
    F.fvv_refine_init(ctx, F.fvv_refine_default_cfg(widths=widths, z_far=Z_FAR))
    return ctx


@pytest.mark.parametrize("widths", [(32, 64, 128), (48, 96, 192)])
def test_e4m3_forward_matches_quantised_oracle(widths):
    import torch
    F = lib()
    ctx = _net(F, widths)
    try:
        rng = np.random.default_rng(11)
        p = U.init_params(widths, seed=6, out_scale=0.5)
        for k in p:
            if k.endswith(".b"):
                p[k] = rng.standard_normal(p[k].shape) * 0.05
        F.fvv_refine_set(ctx, F.FVV_REFINE_PARAMS, _flat(p))
        p32 = {k: v.astype(np.float32).astype(np.float64) for k, v in p.items()}
        n, h, w = 2, 32, 136
        host, dev = _batch(rng, n, h, w)
        x, rgb, _ = _oracle_inputs(host)
        x = U.features(host["rgb"], host["depth"], host["hole"], host["top3"], Z_FAR)
        pred_bf, cache = U.forward(p32, x, rgb)
        scales = U.activation_scales(cache)
        F.fvv_refine_quantize(ctx, None, scales.astype(np.float32))
        assert F.fvv_refine_get_precision(ctx)[0] == F.FVV_PREC_E4M3
        b = F.refine_batch(n, h, w, dev["rgb"], dev["depth"], dev["hole"], dev["top3"])
        out = torch.zeros((n, h, w, 3), dtype=torch.float32, device="cuda")
        out8 = torch.zeros((n, h, w, 3), dtype=torch.uint8, device="cuda")
        F.fvv_refine_forward(ctx, b, out8, out)
        got = out.double().cpu().numpy()
        s32 = scales.astype(np.float32).astype(np.float64)
        ref = U.forward_e4m3(p32, x, rgb, s32)
        base = np.clip(rgb, 0, 1)

        def rel(a, b):
            return np.linalg.norm((a - base) - (b - base)) / np.linalg.norm(b - base)
        spread = max(rel(U.forward_e4m3(p32, x, rgb, s32 * (1 + 1e-6)), ref),
                     rel(U.forward_e4m3(p32, x, rgb, s32 * (1 - 1e-6)), ref), 0.01)
        assert rel(got, ref) <= 3.0 * spread, (rel(got, ref), spread)
        q_gpu, q_ref = rel(got, pred_bf), rel(ref, pred_bf)
        assert 0.75 * q_ref <= q_gpu <= 1.25 * q_ref, (q_gpu, q_ref)
        # the bytes are the rounded float output
        assert np.array_equal(out8.cpu().numpy(), np.floor(got.astype(np.float32) * 255.0 + 0.5).astype(np.uint8))
    finally:
        F.fvv_destroy(ctx)


def test_precision_switch_and_invalidation():
    import torch
    F = lib()
    ctx = _net(F, (32, 64, 128))
    try:
        rng = np.random.default_rng(3)
        n, h, w = 2, 32, 64
        host, dev = _batch(rng, n, h, w)
        b = F.refine_batch(n, h, w, dev["rgb"], dev["depth"], dev["hole"], dev["top3"], dev["target"])
        o_bf = torch.zeros((n, h, w, 3), dtype=torch.uint8, device="cuda")
        F.fvv_refine_forward(ctx, b, o_bf)
        with pytest.raises(F.FvvError) as e:
            F.fvv_refine_set_precision(ctx, F.FVV_PREC_E4M3)        # nothing quantised yet
        assert e.value.code == F.FVV_ERR_STATE
        F.fvv_refine_quantize(ctx, b)                                 # calibrate on the batch
        prec, sc = F.fvv_refine_get_precision(ctx)
        assert prec == F.FVV_PREC_E4M3 and np.all(sc > 0)
        o_q = torch.zeros_like(o_bf)
        F.fvv_refine_forward(ctx, b, o_q)
        assert np.abs(o_q.cpu().numpy().astype(int) - o_bf.cpu().numpy().astype(int)).mean() < 3.0
        F.fvv_refine_set_precision(ctx, F.FVV_PREC_BF16)
        o_b2 = torch.zeros_like(o_bf)
        F.fvv_refine_forward(ctx, b, o_b2)
        assert torch.equal(o_b2, o_bf)
        F.fvv_refine_set_precision(ctx, F.FVV_PREC_E4M3)
        F.fvv_refine_train_step(ctx, b, 1e-3)                         # weights change: back to bf16
        assert F.fvv_refine_get_precision(ctx)[0] == F.FVV_PREC_BF16
        with pytest.raises(F.FvvError):
            F.fvv_refine_set_precision(ctx, F.FVV_PREC_E4M3)
    finally:
        F.fvv_destroy(ctx)
