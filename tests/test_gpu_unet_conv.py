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
                                          (96, 32, 3, 100), (128, 192, 2, 131), (64, 96, 2, 64)])
@pytest.mark.parametrize("relu", [0, 1])
def test_conv3x3_matches_oracle(cin, cout, h, w, relu):
    import torch
    F = lib()
    rng = np.random.default_rng(cin * 7 + cout + h + w)
    n = 2
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
