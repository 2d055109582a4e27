"""CPU oracle of the joint bilateral depth pre-filter of the view-synthesis
side (Sec. VI: a colour-guided joint bilateral filter fills small gaps in
the live depth, in particular along object boundaries).

TEST INFRASTRUCTURE ONLY (tests, smoke check, benchmark CPU leg).  numpy,
FP32 arithmetic in the order stated below.

The paper names the filter but prints neither its window nor its weights.
Readings taken here:

* J1 (what it fills): a pixel without depth (code 0) is filled; every other
  pixel keeps its code.  Depth codes in [d_lo, d_hi] are the sources; the
  background signal 65535 and codes outside the range are neither sources
  nor filled.
* J2 (window and weights): the (2r+1) x (2r+1) window around p, the
  neighbours q in row-major order (dy = -r..r, then dx = -r..r), skipping
  those outside the image and those that are not sources.  The weight is a
  spatial Gaussian times a colour Gaussian of each RGB channel:
  w = ((s[dy, dx] * c[|dR|]) * c[|dG|]) * c[|dB|] with
  s[dy, dx] = exp(-(dx^2 + dy^2) / (2 sigma_s^2)) and
  c[t] = exp(-t^2 / (2 sigma_c^2)), both evaluated in FP64 and rounded to
  FP32 once, and the products taken in FP32.
* J3 (the estimate): acc = acc + w * d and wsum = wsum + w in FP32, in the
  window order; the code is floor(acc / wsum + 0.5), clamped to
  [d_lo, d_hi].
* J4 (support): p is filled only when at least ``min_valid`` neighbours
  are sources and wsum > 0; otherwise it keeps code 0.
* J5: one pass, out of place (every estimate reads the unfiltered frame).
"""
from __future__ import annotations

import numpy as np

DEPTH_BG = 65535


def spatial_table(radius: int, sigma_s: float) -> np.ndarray:
    """s[dy + r, dx + r] in FP32 (J2)."""
    o = np.arange(-radius, radius + 1, dtype=np.float64)
    d2 = o[:, None] ** 2 + o[None, :] ** 2
    return np.exp(-d2 / (2.0 * sigma_s * sigma_s)).astype(np.float32)


def colour_table(sigma_c: float) -> np.ndarray:
    """c[t], t = 0..255, in FP32 (J2)."""
    t = np.arange(256, dtype=np.float64)
    return np.exp(-t * t / (2.0 * sigma_c * sigma_c)).astype(np.float32)


def jbf(depth, rgb, radius: int = 3, sigma_s: float = 2.0, sigma_c: float = 10.0,
        d_lo: int = 1, d_hi: int = 65534, min_valid: int = 3) -> np.ndarray:
    """One pass of the filter over one camera's frame: ``depth`` (H, W)
    uint16 codes, ``rgb`` (H, W, 3) uint8 guidance.  Returns the filtered
    uint16 codes."""
    d = np.asarray(depth, dtype=np.uint16)
    c = np.asarray(rgb, dtype=np.int32)
    H, W = d.shape
    s_tab = spatial_table(radius, sigma_s)
    c_tab = colour_table(sigma_c)
    src = (d >= d_lo) & (d <= d_hi) & (d != DEPTH_BG)
    target = d == 0
    acc = np.zeros((H, W), np.float32)
    wsum = np.zeros((H, W), np.float32)
    count = np.zeros((H, W), np.int32)
    ys, xs = np.nonzero(target)
    for dy in range(-radius, radius + 1):
        for dx in range(-radius, radius + 1):
            qy, qx = ys + dy, xs + dx
            inside = (qy >= 0) & (qy < H) & (qx >= 0) & (qx < W)
            qyc, qxc = np.clip(qy, 0, H - 1), np.clip(qx, 0, W - 1)
            ok = inside & src[qyc, qxc]
            diff = np.abs(c[ys, xs] - c[qyc, qxc])
            w = np.float32(s_tab[dy + radius, dx + radius]) * c_tab[diff[:, 0]]
            w = (w * c_tab[diff[:, 1]]).astype(np.float32)
            w = (w * c_tab[diff[:, 2]]).astype(np.float32)
            dq = d[qyc, qxc].astype(np.float32)
            a = acc[ys, xs]
            ws = wsum[ys, xs]
            acc[ys, xs] = np.where(ok, a + (w * dq).astype(np.float32), a).astype(np.float32)
            wsum[ys, xs] = np.where(ok, ws + w, ws).astype(np.float32)
            count[ys, xs] += ok
    out = d.copy()
    a, ws, n = acc[ys, xs], wsum[ys, xs], count[ys, xs]
    fill = (n >= min_valid) & (ws > 0)
    with np.errstate(divide="ignore", invalid="ignore"):
        v = np.floor((a / np.where(fill, ws, np.float32(1))).astype(np.float32) + np.float32(0.5))
    v = np.clip(v, d_lo, d_hi)
    out[ys[fill], xs[fill]] = v[fill].astype(np.uint16)
    return out
