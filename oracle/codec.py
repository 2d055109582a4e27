"""CPU oracle of the depth codec of the transmission chain (Sec. IV-A, V-A).

TEST INFRASTRUCTURE ONLY (tests, smoke check, benchmark CPU leg).  FP64
numpy, each step written from the paper:

* Eq. (1), depth correction at the capture side: z_post = (alpha z + beta) z
  (z in metres).
* Eq. (2), 12-bit disparity: Y = (2^12 - 3) (1/z - 1/z_far) / (1/z_near -
  1/z_far) + 2 for z in [z_near, z_far]; code 0 is reserved for background
  pixels and code 1 for values out of that range, including pixels without
  depth.
* Eq. (3) and the bit re-arrangement onto 8-bit YUV420: per 2x2 block, the
  8 LSBs of each pixel become its Y value, complemented (255 - LSB) when the
  pixel's 4 MSBs are odd; the 4 MSBs of the top pixels (1,1), (1,2) are
  bit-interleaved into U, those of the bottom pixels (2,1), (2,2) into V.

Readings where the paper is silent (the interleave figure is missing from
the text): Eq. (2) rounds half up, Y = floor(value + 0.5); the interleave
puts bit i of the first pixel's MSBs at bit 2i and bit i of the second
pixel's at bit 2i + 1; the decoder inverts Eq. (2) as
z = 1 / (1/z_far + (Y - 2) (1/z_near - 1/z_far) / 4093), in that order, and
returns depth codes floor(z / unit + 0.5) clamped to [1, 65534]; code 1
decodes to depth code 0 (no depth) and code 0 to 65535, the 16-bit
background signal (a BG pixel has no transmitted depth; the view-synthesis
side takes its depth from the static background model).  Depth code 0 (no
depth) encodes to 1 and the background signal 65535 to 0.
"""
from __future__ import annotations

import numpy as np

Y_LEVELS = 2 ** 12 - 3          # 4093: steps between z_far (Y = 2) and z_near (Y = 4095)
DEPTH_BG = 65535                # 16-bit background signal (12-bit code 0)


def correct(z, alpha, beta):
    """Eq. (1): corrected depth, metres."""
    z = np.asarray(z, np.float64)
    return (alpha * z + beta) * z


def quantize(z, z_near, z_far):
    """Eq. (2): 12-bit disparity codes of depths z (metres); 1 outside
    [z_near, z_far] and for non-positive z."""
    z = np.asarray(z, np.float64)
    inv_n, inv_f = 1.0 / z_near, 1.0 / z_far
    with np.errstate(divide="ignore", invalid="ignore"):
        v = Y_LEVELS * (1.0 / z - inv_f) / (inv_n - inv_f) + 2.0
    y = np.floor(v + 0.5)
    ok = (z >= z_near) & (z <= z_far)
    return np.where(ok, y, 1).astype(np.int64)


def dequantize(y, z_near, z_far):
    """Inverse of Eq. (2): depth in metres of codes y >= 2 (NaN for 0, 1)."""
    y = np.asarray(y, np.float64)
    inv_n, inv_f = 1.0 / z_near, 1.0 / z_far
    z = 1.0 / (inv_f + (y - 2.0) * (inv_n - inv_f) / Y_LEVELS)
    return np.where(y >= 2, z, np.nan)


def encode_table(z_near, z_far, alpha, beta, unit_m):
    """12-bit code of every uint16 depth code d (d = 0: no depth)."""
    d = np.arange(65536, dtype=np.float64)
    y = quantize(correct(d * unit_m, alpha, beta), z_near, z_far)
    y[0] = 1
    y[DEPTH_BG] = 0
    return y


def decode_table(z_near, z_far, unit_m):
    """uint16 depth code of every 12-bit code (0 for code 1, the background
    signal for code 0)."""
    y = np.arange(4096)
    z = dequantize(y, z_near, z_far)
    with np.errstate(invalid="ignore"):
        d = np.clip(np.floor(z / unit_m + 0.5), 1, DEPTH_BG - 1)
    d = np.where(y >= 2, d, 0)
    d[0] = DEPTH_BG
    return d.astype(np.int64)


def _interleave(a, b):
    """Byte with bit 2i = bit i of a and bit 2i + 1 = bit i of b (a, b < 16)."""
    out = np.zeros(np.shape(a), np.int64)
    for i in range(4):
        out |= ((np.asarray(a) >> i) & 1) << (2 * i)
        out |= ((np.asarray(b) >> i) & 1) << (2 * i + 1)
    return out


def _deinterleave(u):
    u = np.asarray(u, np.int64)
    a = np.zeros(u.shape, np.int64)
    b = np.zeros(u.shape, np.int64)
    for i in range(4):
        a |= ((u >> (2 * i)) & 1) << i
        b |= ((u >> (2 * i + 1)) & 1) << i
    return a, b


def pack_yuv420(y12):
    """12-bit map (H x W, both even) -> (Y [H][W], U [H/2][W/2], V [H/2][W/2]) uint8."""
    y12 = np.asarray(y12, np.int64)
    msb, lsb = y12 >> 8, y12 & 255
    Y = np.where(msb % 2 == 0, lsb, 255 - lsb)
    U = _interleave(msb[0::2, 0::2], msb[0::2, 1::2])
    V = _interleave(msb[1::2, 0::2], msb[1::2, 1::2])
    return Y.astype(np.uint8), U.astype(np.uint8), V.astype(np.uint8)


def unpack_yuv420(Y, U, V):
    """Inverse of pack_yuv420."""
    Y = np.asarray(Y, np.int64)
    h, w = Y.shape
    msb = np.zeros((h, w), np.int64)
    msb[0::2, 0::2], msb[0::2, 1::2] = _deinterleave(U)
    msb[1::2, 0::2], msb[1::2, 1::2] = _deinterleave(V)
    lsb = np.where(msb % 2 == 0, Y, 255 - Y)
    return (msb << 8) | lsb


def encode(depth, z_near, z_far, alpha, beta, unit_m):
    """uint16 depth codes (H x W) -> YUV420 planes."""
    return pack_yuv420(encode_table(z_near, z_far, alpha, beta, unit_m)[np.asarray(depth, np.int64)])


def decode(Y, U, V, z_near, z_far, unit_m):
    """YUV420 planes -> uint16 depth codes (0 = no depth, 65535 = background)."""
    return decode_table(z_near, z_far, unit_m)[unpack_yuv420(Y, U, V)].astype(np.uint16)
