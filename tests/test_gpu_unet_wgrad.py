"""Weight and bias gradients of a 3x3 convolution on the tensor cores
(fvv_unet_wgrad3x3) against the FP64 oracle (oracle/unet.py,
conv3x3_backward) on the same bf16 operands.

Products of two bf16 values are exact in fp32, so the only error is the fp32
accumulation over the pixels.  The bound is stated against the sum of the
absolute terms (the oracle's gradient of |x| and |dz|): 2^-12 of it, far
below the error of a wrong tap, shift or channel (of the order of the result
itself).  The result must also be reproducible bit for bit."""
import numpy as np
import pytest

from oracle import unet as U
from fvv_helpers import lib

pytestmark = pytest.mark.gpu


def _bf16(rng, shape):
    import torch
    return torch.from_numpy(rng.standard_normal(shape).astype(np.float32)).to(torch.bfloat16)


# (n, h, w, cin, xstride, cout)
CASES = [
    (2, 5, 40, 8, 8, 32),           # input features: 8 channels in 16 bytes per pixel
    (2, 5, 40, 8, 32, 32),          # 8 of 32 channels per pixel, 32-wide boxes
    (2, 4, 130, 32, 32, 32),        # ragged 64-pixel boxes along a row
    (1, 3, 64, 32, 40, 64),         # pixel stride of 40 channels
    (2, 6, 20, 64, 64, 128),        # narrow image: 16 x 4 pixel boxes
    (1, 2, 100, 96, 96, 32),
    (1, 3, 33, 192, 192, 64),
    (2, 2, 70, 48, 48, 96),         # the wide network's widths
    (1, 2, 64, 144, 144, 48),
    (1, 1, 8, 16, 16, 192),         # 8 x 8 boxes; two tiles of output channels
    (3, 7, 9, 24, 24, 40),          # channel counts that are not multiples of 32
    (4, 32, 128, 64, 64, 64),       # several chunks per CTA
    (8, 128, 128, 32, 32, 32),      # the training crop at level 1: the stages wrap many times
]


@pytest.mark.parametrize("n,h,w,cin,xstride,cout", CASES)
def test_wgrad_matches_oracle(n, h, w, cin, xstride, cout):
    import torch
    F = lib()
    rng = np.random.default_rng(n * 1000 + h * 100 + w + cin * 7 + cout)
    x = _bf16(rng, (n, h, w, xstride))               # channels >= cin: values the kernel must ignore
    dz = _bf16(rng, (n, h, w, cout))
    dw = torch.full((cout, 3, 3, cin), float("nan"), device="cuda")
    db = torch.full((cout,), float("nan"), device="cuda")
    F.fvv_unet_wgrad3x3(x.cuda(), n, h, w, cin, xstride, dz.cuda(), cout, dw, db)
    xd = x[..., :cin].double().numpy()
    dzd = dz.double().numpy()
    zero = np.zeros((cout, 3, 3, cin))
    _, ref_w, ref_b = U.conv3x3_backward(xd, zero, dzd)
    _, abs_w, abs_b = U.conv3x3_backward(np.abs(xd), zero, np.abs(dzd))
    got_w, got_b = dw.double().cpu().numpy(), db.double().cpu().numpy()
    assert np.all(np.isfinite(got_w)) and np.all(np.isfinite(got_b))
    ew = np.abs(got_w - ref_w)
    assert np.all(ew <= 2.0 ** -12 * abs_w + 1e-6), float((ew / (abs_w + 1e-6)).max())
    assert np.all(np.abs(got_b - ref_b) <= 2.0 ** -12 * abs_b + 1e-6)
    assert np.linalg.norm(got_w - ref_w) <= 1e-4 * np.linalg.norm(ref_w)


def test_wgrad_is_reproducible():
    import torch
    F = lib()
    rng = np.random.default_rng(7)
    n, h, w, cin, cout = 4, 64, 128, 96, 32
    x = _bf16(rng, (n, h, w, cin)).cuda()
    dz = _bf16(rng, (n, h, w, cout)).cuda()
    outs = []
    for _ in range(3):
        dw = torch.zeros((cout, 3, 3, cin), device="cuda")
        db = torch.zeros((cout,), device="cuda")
        F.fvv_unet_wgrad3x3(x, n, h, w, cin, 0, dz, cout, dw, db)
        outs.append((dw, db))
    for dw, db in outs[1:]:
        assert torch.equal(dw, outs[0][0]) and torch.equal(db, outs[0][1])


def test_wgrad_rejects_bad_shapes():
    import torch
    F = lib()
    x = torch.zeros((1, 2, 16, 32), dtype=torch.bfloat16, device="cuda")
    dz = torch.zeros((1, 2, 16, 32), dtype=torch.bfloat16, device="cuda")
    dw = torch.zeros((32, 3, 3, 32), device="cuda")
    for args in ((x, 1, 2, 16, 12, 0, dz, 32), (x, 1, 2, 16, 32, 24, dz, 32), (x, 1, 2, 16, 32, 0, dz, 30)):
        with pytest.raises(F.FvvError) as e:
            F.fvv_unet_wgrad3x3(*args, dw, None)
        assert e.value.code == F.FVV_ERR_INVALID_ARG
