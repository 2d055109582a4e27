"""The convolution with the 2x2 max pooling fused into its epilogue (the
encoder's conv + pool pair of the refinement network).  The convolution
output must be bit-identical to the plain convolution's, and the pooled
tensor and window positions must equal the oracle's max pooling
(oracle/unet.py maxpool2: first maximum wins) applied to that output, over
the floor(h/2) x floor(w/2) windows: ragged tiles, odd sizes and several
images included."""
import numpy as np
import pytest

from oracle import unet as U
from fvv_helpers import lib

pytestmark = pytest.mark.gpu


def _bf16(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(torch.bfloat16)


def _pool_ref(y):
    """Oracle pooling of y [n][h][w][c] over the whole windows."""
    n, h, w, c = y.shape
    return U.maxpool2(y[:, :h - h % 2, :w - w % 2])


SHAPES = [(32, 32, 2, 6, 300), (64, 64, 1, 4, 128), (32, 64, 2, 10, 333), (48, 48, 1, 6, 200),
          (16, 48, 2, 5, 131), (8, 32, 1, 9, 257), (96, 32, 1, 3, 2), (32, 64, 3, 7, 1)]


@pytest.mark.parametrize("cin,cout,n,h,w", SHAPES)
def test_conv_pool_bf16(cin, cout, n, h, w):
    import torch
    F = lib()
    rng = np.random.default_rng(cin + 3 * cout + 7 * h + w)
    xb = _bf16(rng.standard_normal((n, h, w, cin))).cuda()
    wb = _bf16(rng.standard_normal((cout, 3, 3, cin)) / np.sqrt(9 * cin)).cuda()
    b = torch.from_numpy(rng.standard_normal(cout).astype(np.float32) * 0.1).cuda()
    y0 = torch.zeros((n, h, w, cout), dtype=torch.bfloat16, device="cuda")
    F.fvv_unet_conv3x3(xb, n, h, w, cin, wb, b, cout, 1, None, y0)
    y = torch.full((n, h, w, cout), -1.0, dtype=torch.bfloat16, device="cuda")
    h2, w2 = h // 2, w // 2
    p = torch.full((n, max(h2, 1), max(w2, 1), cout), -7.0, dtype=torch.bfloat16, device="cuda")
    a = torch.full((n, max(h2, 1), max(w2, 1), cout), 9, dtype=torch.uint8, device="cuda")
    F.fvv_unet_conv3x3_pool(xb, n, h, w, cin, wb, b, cout, y, p, a)
    torch.cuda.synchronize()
    assert torch.equal(y.view(torch.int16), y0.view(torch.int16))
    if h2 == 0 or w2 == 0:                       # no whole window: nothing pooled
        assert (p.float() == -7.0).all() and (a == 9).all()
        return
    ref, arg = _pool_ref(y.float().cpu().numpy().astype(np.float64))
    assert np.array_equal(p.float().cpu().numpy(), ref)
    assert np.array_equal(a.cpu().numpy(), arg)


def test_conv_pool_ties_take_the_first_window_position():
    """A constant input gives equal values in every window: position 0."""
    import torch
    F = lib()
    n, h, w, cin, cout = 1, 4, 140, 32, 32
    x = torch.ones((n, h, w, cin), dtype=torch.bfloat16, device="cuda")
    wt = torch.zeros((cout, 3, 3, cin), dtype=torch.bfloat16, device="cuda")
    b = torch.full((cout,), 0.5, dtype=torch.float32, device="cuda")
    y = torch.zeros((n, h, w, cout), dtype=torch.bfloat16, device="cuda")
    p = torch.zeros((n, 2, 70, cout), dtype=torch.bfloat16, device="cuda")
    a = torch.full((n, 2, 70, cout), 9, dtype=torch.uint8, device="cuda")
    F.fvv_unet_conv3x3_pool(x, n, h, w, cin, wt, b, cout, y, p, a)
    torch.cuda.synchronize()
    assert (p.float() == 0.5).all() and (a == 0).all()


@pytest.mark.parametrize("cin,cout,n,h,w", [(32, 32, 2, 6, 300), (64, 64, 1, 4, 130), (16, 48, 2, 5, 131)])
def test_conv_pool_e4m3(cin, cout, n, h, w):
    import torch
    F = lib()
    rng = np.random.default_rng(11 + cin + cout + w)
    xq = torch.from_numpy(U.e4m3_encode(U.e4m3_round(rng.standard_normal((n, h, w, cin)) * 4))).cuda()
    wq = torch.from_numpy(U.e4m3_encode(U.e4m3_round(rng.standard_normal((cout, 3, 3, cin)) * 8))).cuda()
    b = torch.from_numpy(rng.standard_normal(cout).astype(np.float32) * 0.1).cuda()
    acc, inv = 1.0 / (32.0 * 9 * cin) ** 0.5, 8.0
    y0 = torch.zeros((n, h, w, cout), dtype=torch.uint8, device="cuda")
    F.fvv_unet_conv3x3_e4m3(xq, n, h, w, cin, wq, b, cout, 1, acc, inv, y0)
    y = torch.zeros_like(y0)
    p = torch.zeros((n, h // 2, w // 2, cout), dtype=torch.uint8, device="cuda")
    F.fvv_unet_conv3x3_pool(xq, n, h, w, cin, wq, b, cout, y, p, None, e4m3=True, acc_scale=acc,
                            out_inv_scale=inv)
    torch.cuda.synchronize()
    assert torch.equal(y, y0)
    codes = y.cpu().numpy()
    vals = U.e4m3_decode(codes)
    assert (vals >= 0).all()
    _, arg = _pool_ref(vals)
    h2, w2 = h // 2, w // 2
    win = np.stack([codes[:, 0:2 * h2:2, 0:2 * w2:2], codes[:, 0:2 * h2:2, 1:2 * w2:2],
                    codes[:, 1:2 * h2:2, 0:2 * w2:2], codes[:, 1:2 * h2:2, 1:2 * w2:2]], axis=0)
    ref = np.take_along_axis(win, arg[None], axis=0)[0]
    assert np.array_equal(p.cpu().numpy(), ref)


def test_conv_pool_errors():
    import torch
    F = lib()
    x = torch.zeros((1, 4, 8, 32), dtype=torch.bfloat16, device="cuda")
    wt = torch.zeros((96, 3, 3, 32), dtype=torch.bfloat16, device="cuda")
    y = torch.zeros((1, 4, 8, 96), dtype=torch.bfloat16, device="cuda")
    p = torch.zeros((1, 2, 4, 96), dtype=torch.bfloat16, device="cuda")
    a = torch.zeros((1, 2, 4, 96), dtype=torch.uint8, device="cuda")
    with pytest.raises(F.FvvError) as e:                     # cout 96: one output row per tile
        F.fvv_unet_conv3x3_pool(x, 1, 4, 8, 32, wt, None, 96, y, p, a)
    assert e.value.code == F.FVV_ERR_INVALID_ARG
    with pytest.raises(F.FvvError) as e:                     # window positions are bf16 only
        F.fvv_unet_conv3x3_pool(x, 1, 4, 8, 32, wt, None, 32, y, p, a, e4m3=True)
    assert e.value.code == F.FVV_ERR_INVALID_ARG
    with pytest.raises(F.FvvError) as e:                     # host memory
        F.fvv_unet_conv3x3_pool(x, 1, 4, 8, 32, wt, None, 32, y, np.zeros(64, np.uint16), None)
    assert e.value.code == F.FVV_ERR_INVALID_ARG
