"""The tensor-core 3x3 convolution against the FP64 oracle (oracle/unet.py),
on bf16-rounded inputs: fp32 accumulation then one bf16 rounding, so the
error bound is the output rounding (2^-8 relative) plus a small absolute
term for cancellation."""
import numpy as np
import pytest

from oracle import unet as U
from fvv_helpers import lib

pytestmark = pytest.mark.gpu


def _bf16(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(torch.bfloat16)


@pytest.mark.parametrize("cin,cout,h,w", [(32, 32, 3, 130), (32, 64, 2, 128), (64, 64, 4, 70),
                                          (64, 128, 2, 257), (128, 128, 2, 128), (192, 64, 2, 140),
                                          (96, 32, 3, 100), (128, 192, 2, 131), (64, 96, 2, 64),
                                          (16, 48, 3, 129), (48, 48, 2, 200), (144, 48, 2, 100),
                                          (288, 96, 2, 130), (48, 192, 1, 40), (8, 32, 3, 150),
                                          (8, 48, 2, 64), (24, 64, 2, 100)])
@pytest.mark.parametrize("relu", [0, 1])
def test_conv3x3_matches_oracle(cin, cout, h, w, relu):
    _check_conv(cin, cout, 2, h, w, relu)


# many tiles per CTA: the persistent loop, both TMEM accumulators and the
# stage ring wrap several times; resident and streamed weights
@pytest.mark.parametrize("cin,cout,n,h,w", [(32, 32, 3, 64, 300), (64, 128, 2, 48, 256),
                                            (128, 128, 2, 40, 256), (192, 64, 2, 60, 130),
                                            (48, 96, 2, 50, 640), (8, 32, 3, 64, 300), (8, 48, 2, 50, 200)])
def test_conv3x3_many_tiles(cin, cout, n, h, w):
    _check_conv(cin, cout, n, h, w, 1)


def _check_conv(cin, cout, n, h, w, relu):
    import torch
    F = lib()
    rng = np.random.default_rng(cin * 7 + cout + h + w)
    xb = _bf16(rng.standard_normal((n, h, w, cin)))
    wb = _bf16(rng.standard_normal((cout, 3, 3, cin)) / np.sqrt(9 * cin))
    b = torch.from_numpy(rng.standard_normal(cout).astype(np.float32) * 0.1)
    y = torch.zeros((n, h, w, cout), dtype=torch.bfloat16, device="cuda")
    F.fvv_unet_conv3x3(xb.cuda(), n, h, w, cin, wb.cuda(), b.cuda(), cout, relu, None, y)
    ref = U.conv3x3(xb.double().numpy(), wb.double().numpy(), b.double().numpy())
    if relu:
        ref = np.maximum(ref, 0)
    got = y.float().cpu().numpy()
    err = np.abs(got - ref)
    assert np.all(err <= 2.0 ** -8 * np.abs(ref) + 1e-3), float(err.max())


def test_conv3x3_mask():
    import torch
    F = lib()
    rng = np.random.default_rng(9)
    n, h, w, cin, cout = 1, 3, 140, 64, 32
    xb = _bf16(rng.standard_normal((n, h, w, cin)))
    wb = _bf16(rng.standard_normal((cout, 3, 3, cin)) / 24)
    mask = _bf16(rng.standard_normal((n, h, w, cout)))
    y = torch.zeros((n, h, w, cout), dtype=torch.bfloat16, device="cuda")
    F.fvv_unet_conv3x3(xb.cuda(), n, h, w, cin, wb.cuda(), None, cout, 0, mask.cuda(), y)
    ref = U.conv3x3(xb.double().numpy(), wb.double().numpy(), np.zeros(cout))
    ref = ref * (mask.float().numpy() > 0)
    got = y.float().cpu().numpy()
    assert np.all(np.abs(got - ref) <= 2.0 ** -8 * np.abs(ref) + 1e-3)
    assert np.all(got[mask.float().numpy() <= 0] == 0)


def test_conv3x3_rejects_misaligned_pointers():
    import torch
    F = lib()
    n, h, w, cin, cout = 1, 2, 16, 32, 32
    x = torch.zeros((n, h, w, cin), dtype=torch.bfloat16, device="cuda")
    wt = torch.zeros((cout, 3, 3, cin), dtype=torch.bfloat16, device="cuda")
    b = torch.zeros(cout + 1, device="cuda")
    y = torch.zeros((n, h, w, cout), dtype=torch.bfloat16, device="cuda")
    with pytest.raises(F.FvvError) as e:
        F.fvv_unet_conv3x3(x, n, h, w, cin, wt, b[1:], cout, 1, None, y)
    assert e.value.code == F.FVV_ERR_INVALID_ARG


# ---- FP8 (E4M3) form ---------------------------------------------------------
def _e4m3_ulp(v):
    """Spacing of E4M3 values at |v| (2^-9 in the subnormal range)."""
    _, ex = np.frexp(np.abs(v))
    return np.ldexp(1.0, np.clip(ex - 1, -6, 8) - 3)


@pytest.mark.parametrize("cin,cout,h,w", [(16, 32, 3, 130), (16, 32, 2, 256), (16, 48, 4, 70), (32, 48, 2, 200), (48, 96, 2, 140),
                                          (64, 64, 3, 100), (96, 192, 2, 64), (144, 48, 2, 130),
                                          (288, 96, 2, 128), (192, 192, 1, 140), (64, 128, 40, 256)])
@pytest.mark.parametrize("relu", [0, 1])
def test_conv3x3_e4m3_matches_oracle(cin, cout, h, w, relu):
    """Same quantised operands on both sides: the oracle convolves the
    dequantised E4M3 inputs in FP64, then both round the output once to E4M3.
    The GPU accumulates in fp32, so a value within rounding noise of a tie
    may land on the other neighbour: the bound is one E4M3 spacing, and at
    least 99 % of outputs must be the oracle's code exactly."""
    import torch
    F = lib()
    rng = np.random.default_rng(cin * 3 + cout + h * 7 + w + relu)
    n = 2
    x = rng.standard_normal((n, h, w, cin)) * 2.0
    wgt = rng.standard_normal((cout, 3, 3, cin)) / np.sqrt(9 * cin)
    s_x, s_w = np.abs(x).max() / 448.0, np.abs(wgt).max() / 448.0
    xq, wq = U.e4m3_round(x / s_x), U.e4m3_round(wgt / s_w)
    bias = (rng.standard_normal(cout) * 0.1).astype(np.float32)
    ref = U.conv3x3(xq * s_x, wq * s_w, bias.astype(np.float64))
    if relu:
        ref = np.maximum(ref, 0.0)
    s_y = np.abs(ref).max() / 400.0
    xd = torch.from_numpy(U.e4m3_encode(xq)).cuda()
    wd = torch.from_numpy(U.e4m3_encode(wq)).cuda()
    y = torch.zeros((n, h, w, cout), dtype=torch.uint8, device="cuda")
    F.fvv_unet_conv3x3_e4m3(xd, n, h, w, cin, wd, torch.from_numpy(bias).cuda(), cout, relu,
                            float(np.float32(s_x * s_w)), float(np.float32(1.0 / s_y)), y)
    codes = y.cpu().numpy()
    got = U.e4m3_decode(codes)
    want = ref / s_y
    assert np.all(np.isfinite(got))
    assert np.all(np.abs(got - want) <= _e4m3_ulp(want * (1 + 1e-5)) + 1e-9), float(np.abs(got - want).max())
    assert np.mean(codes == U.e4m3_encode(U.e4m3_round(want))) >= 0.99
