"""Pins of the depth-codec oracle (oracle/codec.py) to what the paper and
the arithmetic fix (Sec. IV-A, V-A, Eq. (1)-(3))."""
import numpy as np
import pytest

from oracle import codec as K

ZN, ZF = 0.5, 8.0


def test_eq2_endpoints_and_reserved_codes():
    """Y(z_far) = 2 and Y(z_near) = 2^12 - 1 exactly; outside the range and
    without depth the code is the reserved 1."""
    assert K.quantize(ZF, ZN, ZF) == 2
    assert K.quantize(ZN, ZN, ZF) == 4095
    assert K.quantize(ZF * 1.0001, ZN, ZF) == 1 and K.quantize(ZN * 0.9999, ZN, ZF) == 1
    assert K.quantize(0.0, ZN, ZF) == 1 and K.quantize(-1.0, ZN, ZF) == 1
    # disparity is linear in 1/z: the midpoint of 1/z maps to the middle code
    zm = 1.0 / (0.5 * (1.0 / ZN + 1.0 / ZF))
    assert K.quantize(zm, ZN, ZF) == int(np.floor(4093 / 2 + 2 + 0.5))
    assert np.all(np.diff(K.quantize(np.linspace(ZN, ZF, 5000), ZN, ZF)) <= 0)   # nearer = larger


def test_eq2_inverse_within_half_a_step():
    """Dequantising a code returns a depth whose 1/z lies within half a
    quantisation step of the input's."""
    z = np.random.default_rng(0).uniform(ZN, ZF, 100000)
    zq = K.dequantize(K.quantize(z, ZN, ZF), ZN, ZF)
    step = (1.0 / ZN - 1.0 / ZF) / 4093
    assert np.all(np.abs(1.0 / zq - 1.0 / z) <= 0.5 * step * (1 + 1e-9))
    assert K.dequantize(2, ZN, ZF) == pytest.approx(ZF, rel=1e-15)
    assert K.dequantize(4095, ZN, ZF) == pytest.approx(ZN, rel=1e-15)
    assert np.isnan(K.dequantize(1, ZN, ZF)) and np.isnan(K.dequantize(0, ZN, ZF))


def test_eq1_correction():
    assert K.correct(2.0, 0.0, 1.0) == 2.0
    assert K.correct(2.0, 0.01, 1.0) == pytest.approx((0.02 + 1.0) * 2.0)
    assert K.correct(3.0, -0.02, 1.1) == pytest.approx((1.1 - 0.06) * 3.0)


def test_eq3_removes_the_lsb_discontinuities():
    """Folded Y values of consecutive 12-bit codes differ by at most 1 (the
    8 LSBs alone jump by 255 at every multiple of 256)."""
    v = np.arange(4096).reshape(64, 64)
    Y, _, _ = K.pack_yuv420(v)
    y = Y.reshape(-1).astype(int)
    assert np.max(np.abs(np.diff(y))) == 1
    assert np.max(np.abs(np.diff(v.reshape(-1) & 255))) == 255


def test_interleave_closed_forms():
    """U takes bit i of pixel (1,1)'s 4 MSBs at bit 2i and bit i of pixel
    (1,2)'s at bit 2i + 1; V the same for the bottom row."""
    y12 = np.array([[0xF00, 0x000], [0x000, 0xF00]])
    _, U, V = K.pack_yuv420(y12)
    assert U[0, 0] == 0b01010101 and V[0, 0] == 0b10101010
    y12 = np.array([[0x500, 0xA00], [0x300, 0xC00]])       # 0101, 1010 / 0011, 1100
    _, U, V = K.pack_yuv420(y12)
    assert U[0, 0] == 0b10011001 and V[0, 0] == 0b10100101


@pytest.mark.parametrize("pos", [(0, 0), (0, 1), (1, 0), (1, 1)])
def test_pack_round_trip_every_code_every_position(pos):
    """All 4096 codes at each position of a 2x2 block, with random codes at
    the other three, survive pack + unpack exactly."""
    rng = np.random.default_rng(pos[0] * 2 + pos[1])
    blocks = rng.integers(0, 4096, (4096, 2, 2))
    blocks[:, pos[0], pos[1]] = np.arange(4096)
    y12 = blocks.transpose(1, 0, 2).reshape(2, 4096 * 2)       # 4096 blocks side by side
    assert np.array_equal(K.unpack_yuv420(*K.pack_yuv420(y12)), y12)


def test_depth_round_trip_through_the_codec():
    """encode -> decode returns every in-range depth code to within the
    depth width of half a disparity step; out-of-range and missing depth
    decode to 0; the background signal survives as itself."""
    unit = 0.001
    d = np.arange(65536)
    y = K.encode_table(ZN, ZF, 0.0, 1.0, unit)
    back = K.decode_table(ZN, ZF, unit)[y]
    z = d * unit
    inr = (z >= ZN) & (z <= ZF)
    step = (1.0 / ZN - 1.0 / ZF) / 4093
    tol = 0.5 * step * z * z / unit * 1.0001 + 0.5          # half a step in 1/z, in codes, + rounding
    assert np.all(np.abs(back[inr] - d[inr]) <= tol[inr])
    sig = d == K.DEPTH_BG
    assert np.all(back[~inr & ~sig] == 0) and back[0] == 0
    assert back[K.DEPTH_BG] == K.DEPTH_BG
    Y, U, V = K.encode(d[:4096].reshape(64, 64), ZN, ZF, 0.0, 1.0, unit)
    assert np.array_equal(K.decode(Y, U, V, ZN, ZF, unit), back[:4096].reshape(64, 64))


def test_background_signal_is_code_zero():
    """Eq. (2) reserves code 0 for background pixels and code 1 for pixels
    out of range or without depth: the 16-bit background signal encodes to
    0 and code 0 decodes to it; no depth code decodes to the signal."""
    enc = K.encode_table(ZN, ZF, 0.0, 1.0, 0.001)
    dec = K.decode_table(ZN, ZF, 0.001)
    assert enc[K.DEPTH_BG] == 0 and enc[0] == 1
    assert np.all(enc[1:K.DEPTH_BG] >= 1)
    assert dec[0] == K.DEPTH_BG and dec[1] == 0
    assert np.all((dec[2:] >= 1) & (dec[2:] <= K.DEPTH_BG - 1))
    # a near z_far that reaches the top of the 16-bit range clamps below the signal
    dec_far = K.decode_table(0.5, 70.0, 0.001)
    assert dec_far[2] == K.DEPTH_BG - 1


def test_encoder_applies_the_eq1_correction():
    """The encoder quantises the corrected depth of Eq. (1), not the raw one:
    with alpha = 0 and beta = 2 (corrected z = 2 z) a code d is encoded as
    the uncorrected encoder encodes 2 d; with beta = 1 the two encoders are
    the same."""
    unit = 0.001
    d = np.arange(1, 30000)
    doubled = K.encode_table(ZN, ZF, 0.0, 2.0, unit)
    plain = K.encode_table(ZN, ZF, 0.0, 1.0, unit)
    assert np.array_equal(doubled[d], plain[2 * d])
    assert np.array_equal(K.encode_table(ZN, ZF, 0.0, 1.0, unit), plain)
