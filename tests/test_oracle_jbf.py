"""Pins of the joint bilateral depth pre-filter oracle (oracle/jbf.py,
Sec. VI) against closed forms, brute force and what the filter is for."""
import math

import numpy as np
import pytest

import synthetic as S
from oracle import jbf as J

BG = J.DEPTH_BG


def _holes(rng, H, W, frac, border=0):
    m = rng.random((H, W)) < frac
    if border:
        m[:border] = m[-border:] = False
        m[:, :border] = m[:, -border:] = False
    return m


def test_sources_and_signal_are_untouched():
    rng = np.random.default_rng(0)
    d = rng.integers(1, 9000, (40, 50)).astype(np.uint16)
    d[_holes(rng, 40, 50, 0.1)] = 0
    d[_holes(rng, 40, 50, 0.1)] = BG
    rgb = rng.integers(0, 256, (40, 50, 3)).astype(np.uint8)
    out = J.jbf(d, rgb)
    keep = d != 0
    assert np.array_equal(out[keep], d[keep])
    assert np.all(out[d == 0] != BG)


def test_constant_depth_fills_with_that_depth():
    """A convex combination of equal codes is that code, whatever the colours."""
    rng = np.random.default_rng(1)
    d = np.full((48, 64), 1537, np.uint16)
    h = _holes(rng, 48, 64, 0.15)
    d[h] = 0
    rgb = rng.integers(0, 256, (48, 64, 3)).astype(np.uint8)
    out = J.jbf(d, rgb, radius=2, sigma_c=40.0, min_valid=1)
    filled = out[h] != 0
    assert filled.mean() > 0.95
    assert np.all(out[h][filled] == 1537)


def test_linear_ramp_is_reproduced_by_a_symmetric_window():
    """Uniform colour, a planar depth ramp and isolated holes whose whole
    window is valid: the symmetric spatial weights average a linear function
    to its value at the centre."""
    H, W, r = 40, 60, 3
    y, x = np.mgrid[0:H, 0:W]
    ramp = (2000 + 7 * x + 3 * y).astype(np.uint16)
    d = ramp.copy()
    holes = [(10, 10), (20, 30), (30, 45), (15, 50)]
    for (hy, hx) in holes:
        d[hy, hx] = 0
    rgb = np.full((H, W, 3), 90, np.uint8)
    out = J.jbf(d, rgb, radius=r, sigma_s=2.5)
    for (hy, hx) in holes:
        assert out[hy, hx] == ramp[hy, hx]


@pytest.mark.parametrize("hole_colour,expect", [((200, 30, 30), 1000), ((30, 30, 200), 3000)])
def test_colour_guidance_picks_the_matching_side(hole_colour, expect):
    """Two regions of different colour and depth; a column of holes on their
    boundary takes the depth of the region whose colour it has."""
    H, W = 20, 30
    d = np.where(np.arange(W)[None, :] < 15, 1000, 3000).astype(np.uint16).repeat(H, 0)
    rgb = np.zeros((H, W, 3), np.uint8)
    rgb[:, :15] = (200, 30, 30)
    rgb[:, 15:] = (30, 30, 200)
    d[:, 15] = 0
    rgb[:, 15] = hole_colour
    out = J.jbf(d, rgb, radius=3, sigma_s=2.0, sigma_c=10.0)
    assert np.all(out[3:-3, 15] == expect)


def test_large_sigma_c_is_a_spatial_gaussian_average():
    """With colour weights 1, each filled code is the Gaussian-weighted mean
    of the valid codes in the window (brute force in FP64), to within the
    last unit of the rounding."""
    rng = np.random.default_rng(2)
    H, W, r, ss = 24, 32, 2, 1.7
    d = rng.integers(500, 4000, (H, W)).astype(np.uint16)
    h = _holes(rng, H, W, 0.2)
    d[h] = 0
    rgb = rng.integers(0, 256, (H, W, 3)).astype(np.uint8)
    out = J.jbf(d, rgb, radius=r, sigma_s=ss, sigma_c=1e9, min_valid=1)
    for yy, xx in zip(*np.nonzero(h)):
        num = den = 0.0
        for dy in range(-r, r + 1):
            for dx in range(-r, r + 1):
                qy, qx = yy + dy, xx + dx
                if 0 <= qy < H and 0 <= qx < W and d[qy, qx] != 0:
                    w = math.exp(-(dx * dx + dy * dy) / (2 * ss * ss))
                    num += w * float(d[qy, qx])
                    den += w
        if den == 0.0:
            assert out[yy, xx] == 0
        else:
            assert abs(int(out[yy, xx]) - math.floor(num / den + 0.5)) <= 1


def test_support_rule_and_reach():
    """A hole with fewer than min_valid source neighbours stays empty; a disc
    of holes shrinks by at most the radius per pass."""
    H, W, r = 41, 41, 3
    d = np.full((H, W), 2500, np.uint16)
    y, x = np.mgrid[0:H, 0:W]
    disc = (y - 20) ** 2 + (x - 20) ** 2 <= 10 ** 2
    d[disc] = 0
    rgb = np.full((H, W, 3), 128, np.uint8)
    out = J.jbf(d, rgb, radius=r, min_valid=3)
    still = out == 0
    assert still[20, 20]                                       # the centre is out of reach
    assert np.all(~still[~disc])
    inner = (y - 20) ** 2 + (x - 20) ** 2 <= (10 - r - 1) ** 2
    assert np.all(still[inner])
    assert np.all(out[disc & ~still] == 2500)
    # an isolated source: its neighbours see one valid sample only
    d2 = np.zeros((9, 9), np.uint16)
    d2[4, 4] = 1800
    out2 = J.jbf(d2, np.zeros((9, 9, 3), np.uint8), radius=2, min_valid=2)
    assert np.count_nonzero(out2) == 1
    out3 = J.jbf(d2, np.zeros((9, 9, 3), np.uint8), radius=2, min_valid=1)
    assert np.count_nonzero(out3) == 25 and np.all(out3[2:7, 2:7] == 1800)


def test_filter_closes_holes_of_the_synthesised_view(oracle_mod):
    """The purpose the paper states: with the noisy 9-camera frames
    (dropout discs), pre-filtering every camera's depth leaves fewer holes in
    a synthesised view and brings its depth closer to the analytic ray-cast."""
    wl = S.workload("plain_9cam_1280x720", scale=0.25)
    cams, view = wl["cams"], wl["views"][40]
    filt = np.stack([J.jbf(wl["depth"][k], wl["rgb"][k]) for k in range(len(cams))])
    assert (filt == 0).mean() < 0.7 * (wl["depth"] == 0).mean()
    a = oracle_mod.synthesize(cams, wl["rgb"], wl["depth"], view, wl["look_at"], hole_fill=0)
    b = oracle_mod.synthesize(cams, wl["rgb"], filt, view, wl["look_at"], hole_fill=0)
    assert b["hole"].mean() <= a["hole"].mean()
    gt = S.render(wl["scene"], view)
    z = gt["z"] * 1000.0
    both = (a["hole"] == 0) & (b["hole"] == 0) & np.isfinite(z)
    ea = np.median(np.abs(a["depth"][both] - z[both]) / z[both])
    eb = np.median(np.abs(b["depth"][both] - z[both]) / z[both])
    assert eb <= ea * 1.05


@pytest.mark.parametrize("channel", [0, 1, 2])
def test_each_colour_channel_guides_alone(channel):
    """Two depth regions whose colours differ in one channel only, a column
    of holes between them whose colour is the right region's: every colour
    channel enters the weight on its own, so the holes take the right
    region's depth (the left neighbours' weight carries c(200) ~ e^-200 of
    that channel's colour Gaussian, sigma_c = 10)."""
    H, W = 9, 21
    d = np.zeros((H, W), np.uint16)
    d[:, :10] = 1000
    d[:, 11:] = 3000
    rgb = np.full((H, W, 3), 100, np.uint8)
    rgb[:, :10, channel] = 0
    rgb[:, 10:, channel] = 200
    out = J.jbf(d, rgb, radius=2, sigma_s=2.0, sigma_c=10.0, min_valid=3)
    assert np.all(out[:, 10] == 3000), out[:, 10]
