"""Failure detection without a GPU fault: a bounded wait that nothing
completes gives up after its limit, the kernel exits, the host reads
FVV_ERR_TIMEOUT, and the context keeps working afterwards."""
import time

import numpy as np
import pytest

import synthetic as S
from fvv_helpers import lib, gpu_run

pytestmark = pytest.mark.gpu


def test_wait_that_completes_returns_ok():
    F = lib()
    assert F.fvv_selftest_bounded_wait(True, 20000) == F.FVV_OK


def test_wait_that_nothing_completes_times_out_and_context_survives(oracle_mod):
    import torch
    F = lib()
    F.fvv_selftest_bounded_wait(True, 20000)            # warm the module
    t0 = time.perf_counter()
    st = F.fvv_selftest_bounded_wait(False, 50000)      # 50 ms limit
    el = time.perf_counter() - t0
    assert st == F.FVV_ERR_TIMEOUT
    assert "ran out" in F.fvv_last_error()
    assert 0.04 <= el < 1.5, el
    # a stream of the caller's works the same way
    s = torch.cuda.Stream()
    assert F.fvv_selftest_bounded_wait(False, 10000, s) == F.FVV_ERR_TIMEOUT
    assert F.fvv_selftest_bounded_wait(True, 10000, s) == F.FVV_OK
    torch.cuda.synchronize()
    # the CUDA context is still usable: a synthesis matches the oracle
    wl = S.workload("plain_2cam_320x240")
    v = wl["views"][0]
    got = gpu_run(wl["cams"], wl["rgb"], wl["depth"], [v], wl["look_at"])[0]
    ref = oracle_mod.synthesize(wl["cams"], wl["rgb"], wl["depth"], v, wl["look_at"])
    assert np.array_equal(got["keys"], ref["keys"])
