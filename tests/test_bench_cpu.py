"""Host-side figures the benchmark reports: the refinement network's FLOP
count (the numerator of its tensor-core fraction) against the multiply-adds
the oracle's own forward pass performs, counted by wrapping its convolution
routines."""
import os
import sys

import numpy as np
import pytest

from oracle import unet as U

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


@pytest.mark.parametrize("widths", [(32, 64, 128), (48, 96, 192)])
def test_unet_flops_equal_the_oracle_forward_multiply_adds(widths, monkeypatch):
    macs = [0]
    conv3, conv1 = U.conv3x3, U.conv1x1

    def count3(x, w, b):
        n, h, wd, _ = x.shape
        co, _, _, ci = w.shape
        macs[0] += n * h * wd * co * 9 * ci
        return conv3(x, w, b)

    def count1(x, w, b):
        n, h, wd, _ = x.shape
        co, ci = w.shape
        macs[0] += n * h * wd * co * ci
        return conv1(x, w, b)

    monkeypatch.setattr(U, "conv3x3", count3)
    monkeypatch.setattr(U, "conv1x1", count1)
    H, W = 16, 24
    p = U.init_params(widths, seed=0)
    x = np.random.default_rng(0).standard_normal((1, H, W, 8))
    U.forward(p, x, np.zeros((1, H, W, 3)))
    assert bench.unet_flops(H, W, widths) == 2.0 * macs[0]
