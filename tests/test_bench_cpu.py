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


def _fake_tree(tmp_path, kernels_src, summary):
    """A repository copy holding only what the profile lookups read: the two
    kernel sources the SHA covers and one profile summary."""
    csrc = tmp_path / "paper_2007_00558_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "fvv_kernels.cu").write_text(kernels_src)
    (csrc / "fvv_internal.h").write_text("// header\n")
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "resolve_9cam_1280x720.txt").write_text(summary)
    return str(tmp_path)


def test_profiled_figures_are_gated_by_the_kernel_source_sha(tmp_path, monkeypatch):
    """Traffic and instruction counts from a committed ncu summary are used
    only while the kernel sources still hash to the SHA stored beside them;
    after any change they read as unknown (None)."""
    monkeypatch.setattr(bench, "ROOT", _fake_tree(tmp_path, "// kernels v1\n", ""))
    sha = bench.kernel_source_sha()
    text = "dram_bytes_per_view: 44.0e6\nwarp_instructions_per_view: 32.5e6\nkernel_source_sha: %s\n" % sha
    (tmp_path / "profiles" / "resolve_9cam_1280x720.txt").write_text(text)
    assert bench.profiled_traffic("resolve", 8) == pytest.approx(8 * 44.0e6)
    assert bench.profiled_instructions("resolve") == pytest.approx(32.5e6)
    (tmp_path / "paper_2007_00558_gb300" / "csrc" / "fvv_kernels.cu").write_text("// kernels v2\n")
    assert bench.kernel_source_sha() != sha
    assert bench.profiled_traffic("resolve", 8) is None
    assert bench.profiled_instructions("resolve") is None
    assert bench.profiled_traffic("warp_splat", 8) is None          # no summary at all


def test_issue_roofline_against_schedulers_times_clock(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", _fake_tree(tmp_path, "// k\n", ""))
    text = "warp_instructions_per_view: 10.0e6\nkernel_source_sha: %s\n" % bench.kernel_source_sha()
    (tmp_path / "profiles" / "resolve_9cam_1280x720.txt").write_text(text)
    r = bench.issue_roofline("resolve", 8, 100e-6, 2000.0, 152)
    assert r["peak"] == pytest.approx(152 * 4 * 2000e6)
    assert r["achieved"] == pytest.approx(8 * 10.0e6 / 100e-6)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert bench.issue_roofline("resolve", 8, 100e-6, None, 152) is None   # no clock sample


def test_step_bytes_count_every_kernel_once():
    """The clear's bytes move into the resolve (it empties the next batch's
    z-buffer), so splat + resolve hold the whole step: depth 2 K Ns, atomics
    8 rho K Ns, keys cleared, read and 5 (n_ref - 1) Nd gathered, 6 Nd of
    colour."""
    K, Ns, Nd, rho, n_ref = 9, 921600, 921600, 0.95, 9
    a = bench.algorithmic_bytes(K, Ns, Nd, rho, n_ref)
    step = a["warp_splat"] + a["resolve"]
    assert step == pytest.approx(2 * K * Ns + 8 * rho * K * Ns + 8 * Nd + 8 * Nd + 5 * (n_ref - 1) * Nd + 6 * Nd)
    assert a["clear_keys"] == pytest.approx(8 * Nd)
    assert step / 1e6 == pytest.approx(136.76, abs=0.01)


def test_compulsory_bytes_are_the_frames_read_once_and_the_view_written_once():
    """5 K Ns + 3 Nd: 9 cameras' uint16 depth and RGB8 colour at 1280x720,
    one RGB8 view, 44.2 MB; below the algorithmic bytes of the step."""
    K, Ns, Nd = 9, 921600, 921600
    c = bench.compulsory_bytes(K, Ns, Nd)
    assert c == 9 * 921600 * (2 + 3) + 921600 * 3
    assert c / 1e6 == pytest.approx(44.24, abs=0.01)
    a = bench.algorithmic_bytes(K, Ns, Nd, 0.95, K)
    assert c < a["warp_splat"] + a["resolve"]


def test_recorded_runs_are_read_from_their_json_block(tmp_path, monkeypatch):
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "x.md").write_text("# t\n\n```json\n{\"a\": 1, \"b\": [2, 3]}\n```\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    rec = bench.recorded_run("x.md", "python bench.py --x")
    assert rec["a"] == 1 and rec["b"] == [2, 3]
    assert "python bench.py --x" in rec["source"] and "profiles/x.md" in rec["source"]
    assert bench.recorded_run("missing.md", "c") is None
