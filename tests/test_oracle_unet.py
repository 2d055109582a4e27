"""Pins of the FP64 refinement-network oracle (oracle/unet.py): forward
against an independent library routine and hand cases, backward against
finite differences and adjoint identities."""
import numpy as np
import pytest

from oracle import unet as U

scipy_signal = pytest.importorskip("scipy.signal")


def test_conv3x3_matches_scipy_correlate():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 6, 5, 3))
    w = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    y = U.conv3x3(x, w, b)
    for n in range(2):
        xp = np.pad(x[n], ((1, 1), (1, 1), (0, 0)))
        for co in range(4):
            ref = sum(scipy_signal.correlate2d(xp[..., ci], w[co, :, :, ci], mode="valid")
                      for ci in range(3)) + b[co]
            assert np.allclose(y[n, ..., co], ref, rtol=1e-12, atol=1e-12)


def test_conv1x1_is_channel_matmul():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((1, 3, 4, 5))
    w = rng.standard_normal((2, 5))
    b = rng.standard_normal(2)
    y = U.conv1x1(x, w, b)
    for i in range(3):
        for j in range(4):
            assert np.allclose(y[0, i, j], w @ x[0, i, j] + b)


def _fd(f, arr, idx, eps=1e-6):
    old = arr[idx]
    arr[idx] = old + eps
    fp = f()
    arr[idx] = old - eps
    fm = f()
    arr[idx] = old
    return (fp - fm) / (2 * eps)


def test_conv3x3_backward_finite_differences_and_adjoint():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((1, 5, 4, 3))
    w = rng.standard_normal((2, 3, 3, 3))
    b = rng.standard_normal(2)
    r = rng.standard_normal((1, 5, 4, 2))
    f = lambda: float(np.sum(U.conv3x3(x, w, b) * r))
    dx, dw, db = U.conv3x3_backward(x, w, r)
    for idx in [(0, 0, 0, 0), (0, 4, 3, 2), (0, 2, 1, 1), (0, 0, 3, 1)]:
        assert abs(_fd(f, x, idx) - dx[idx]) < 1e-7
    for idx in [(0, 0, 0, 0), (1, 2, 2, 2), (1, 1, 0, 1)]:
        assert abs(_fd(f, w, idx) - dw[idx]) < 1e-7
    assert abs(_fd(f, b, (1,)) - db[1]) < 1e-7
    # adjoint: <conv(x), r> = <x, conv^T(r)> with zero bias
    y0 = U.conv3x3(x, w, np.zeros(2))
    assert np.isclose(np.sum(y0 * r), np.sum(x * dx))


def test_maxpool_and_upsample():
    x = np.array([[1, 5, 2, 2], [3, 4, 2, 1], [0, 0, 7, 8], [0, 9, 6, 8]], float)[None, :, :, None]
    y, arg = U.maxpool2(x)
    assert y[0, :, :, 0].tolist() == [[5, 2], [9, 8]]
    # ties (2, 2 in the top-right block; 8, 8 bottom-right): first in scan order
    assert arg[0, :, :, 0].tolist() == [[1, 0], [3, 1]]
    d = U.maxpool2_backward(arg, np.array([[10, 20], [30, 40]], float)[None, :, :, None])
    assert d[0, :, :, 0].tolist() == [[0, 10, 20, 0], [0, 0, 0, 0], [0, 0, 0, 40], [0, 30, 0, 0]]
    u = U.up2(np.arange(4.0).reshape(1, 2, 2, 1))
    assert u[0, :, :, 0].tolist() == [[0, 0, 1, 1], [0, 0, 1, 1], [2, 2, 3, 3], [2, 2, 3, 3]]
    rng = np.random.default_rng(3)
    a, r = rng.standard_normal((1, 3, 2, 4)), rng.standard_normal((1, 6, 4, 4))
    assert np.isclose(np.sum(U.up2(a) * r), np.sum(a * U.up2_backward(r)))


def test_network_gradient_finite_differences():
    rng = np.random.default_rng(4)
    p = U.init_params(widths=(3, 4, 5), seed=5, out_scale=0.1)
    for k in p:
        if k.endswith(".b"):
            p[k] = rng.standard_normal(p[k].shape) * 0.1
    x = rng.standard_normal((2, 8, 8, 8))
    rgb = 0.5 + 0.05 * rng.standard_normal((2, 8, 8, 3))
    target = rng.uniform(0.3, 0.7, (2, 8, 8, 3))

    def loss():
        pred, _ = U.forward(p, x, rgb)
        return U.mse(pred, target)[0]

    pred, cache = U.forward(p, x, rgb)
    assert np.all((cache["s"] > 0) & (cache["s"] < 1))
    _, dpred = U.mse(pred, target)
    g = U.backward(p, cache, dpred)
    checked = 0
    for k in p:
        flat = p[k].reshape(-1)
        for j in rng.choice(flat.size, min(3, flat.size), replace=False):
            idx = np.unravel_index(j, p[k].shape)
            num = _fd(loss, p[k], idx, eps=1e-6)
            assert abs(num - g[k][idx]) <= 1e-6 * max(1e-3, abs(num)) + 1e-9, (k, idx, num, g[k][idx])
            checked += 1
    assert checked >= 50


def test_clamp_blocks_gradient_and_zero_net_is_identity():
    p = U.init_params(widths=(2, 2, 2), seed=1)
    for k in p:
        p[k] = np.zeros_like(p[k])
    rgb = np.linspace(-0.2, 1.2, 2 * 4 * 4 * 3).reshape(2, 4, 4, 3)
    x = np.zeros((2, 4, 4, 8))
    pred, cache = U.forward(p, x, rgb)
    assert np.allclose(pred, np.clip(rgb, 0, 1))
    g = U.backward(p, cache, np.ones_like(pred))
    inside = ((rgb > 0) & (rgb < 1)).sum(axis=(0, 1, 2))
    assert np.allclose(g["out.b"], inside)


def test_adam_single_step_closed_form():
    p = {"a": np.array([1.0, -2.0])}
    g = {"a": np.array([0.5, -0.25])}
    st = {}
    U.adam_step(p, g, st, lr=0.1)
    # first bias-corrected step moves by lr * g / (|g| + eps) = lr * sign(g)
    assert np.allclose(p["a"], [1.0 - 0.1, -2.0 + 0.1], atol=1e-6)
    # with a gradient of the order of eps the epsilon shows: the first step
    # is lr g / (sqrt(v) + eps) (eps added after the root), not lr g / sqrt(v + eps)
    p = {"a": np.array([0.0])}
    U.adam_step(p, {"a": np.array([1e-6])}, {}, lr=0.1)
    assert p["a"][0] == pytest.approx(-0.1 * 1e-6 / (1e-6 + 1e-8), rel=1e-9)


def test_e4m3_closed_forms():
    """Values fixed by the format: largest finite 448, smallest subnormal
    2^-9, ties to the even mantissa, saturation, exact round trip of all 254
    finite codes."""
    r = U.e4m3_round
    assert r(448.0) == 448.0 and r(1e6) == 448.0 and r(-1e6) == -448.0
    assert r(464.0) == 448.0                       # tie between 448 (m=6) and 480 (not finite): even m=6
    assert r(2.0 ** -9) == 2.0 ** -9 and r(2.0 ** -10) == 0.0 and r(1.5 * 2.0 ** -9) == 2.0 ** -8
    assert r(1.0625) == 1.0 and r(1.1875) == 1.25  # ties between mantissas 0|1 and 1|2
    assert r(1.0624) == 1.0 and r(1.0626) == 1.125
    assert r(2.0 ** -6) == 2.0 ** -6 and r(0.875 * 2.0 ** -6) == 0.875 * 2.0 ** -6   # normal / subnormal edge
    assert np.signbit(r(-0.0))
    codes = np.array([c for c in range(256) if c not in (0x7F, 0xFF)], np.uint8)
    vals = U.e4m3_decode(codes)
    assert np.all(np.isfinite(vals)) and vals.max() == 448.0
    assert np.array_equal(U.e4m3_round(vals), vals)
    assert np.array_equal(U.e4m3_encode(vals), codes)


def test_e4m3_matches_torch_float8():
    """Rounding and encoding agree byte for byte with PyTorch's float8_e4m3fn
    conversion (round to nearest even; values beyond 448 are saturated first,
    since that conversion does not saturate)."""
    torch = pytest.importorskip("torch")
    if not hasattr(torch, "float8_e4m3fn"):
        pytest.skip("no float8_e4m3fn")
    rng = np.random.default_rng(5)
    x = np.concatenate([rng.standard_normal(20000) * 10.0, rng.standard_normal(20000) * 0.01,
                        np.ldexp(rng.random(20000) + 1.0, rng.integers(-12, 9, 20000)) *
                        np.where(rng.random(20000) < 0.5, -1, 1),
                        np.arange(-480.0, 480.0, 0.125)])
    x = np.clip(x, -448.0, 448.0)
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.float8_e4m3fn)
    ours = U.e4m3_encode(U.e4m3_round(x.astype(np.float32).astype(np.float64)))
    assert np.array_equal(ours, ref.view(torch.uint8).numpy())


def test_forward_e4m3_without_rounding_is_the_network(monkeypatch):
    """With the E4M3 rounding replaced by the identity, the quantised form's
    scale bookkeeping (input and output scales, the concat parts' ratios
    folded into the weights, the accumulator multiplier) must cancel exactly:
    it then equals the plain forward pass."""
    rng = np.random.default_rng(2)
    for widths in ((32, 64, 128), (48, 96, 192)):
        p = U.init_params(widths, seed=4, out_scale=0.5)
        for k in p:
            if k.endswith(".b"):
                p[k] = rng.standard_normal(p[k].shape) * 0.05
        x = rng.random((1, 8, 8, 8))
        rgb = rng.random((1, 8, 8, 3)) * 0.6 + 0.2
        pred, cache = U.forward(p, x, rgb)
        scales = U.activation_scales(cache) * rng.uniform(0.5, 2.0, 10)    # any positive scales
        monkeypatch.setattr(U, "e4m3_round", lambda v: np.asarray(v, np.float64))
        q = U.forward_e4m3(p, x, rgb, scales)
        monkeypatch.undo()
        assert np.allclose(q, pred, rtol=0, atol=1e-12)
        # and with rounding it stays close (3 mantissa bits per tensor)
        q8 = U.forward_e4m3(p, x, rgb, U.activation_scales(cache))
        assert np.abs(q8 - pred).max() < 0.1


def test_features_follow_the_stated_input_layout():
    """The network's 8 input channels are, in this order, the blended RGB,
    the depth, the hole mask and the three largest view weights (the
    refinement's stated input), scaled to [0, 1]: RGB / 255, depth / z_far."""
    rgb = np.array([[[[255, 0, 51]]]], np.uint8)
    depth = np.array([[[2500.0]]], np.float32)
    hole = np.array([[[1]]], np.uint8)
    top3 = np.array([[[[0.5, 0.3, 0.2]]]], np.float32)
    f = U.features(rgb, depth, hole, top3, z_far=10000.0)
    assert f.shape == (1, 1, 1, 8)
    assert np.allclose(f[0, 0, 0], [1.0, 0.0, 0.2, 0.25, 1.0, 0.5, 0.3, 0.2], rtol=0, atol=1e-7)


def test_activation_scales_map_each_maximum_to_448():
    """Per-tensor scaling to the E4M3 range: the largest ReLU output of each
    conv tensor divided by its scale is 448, the largest finite E4M3 value
    (so it is kept, and nothing saturates); an all-zero tensor keeps scale 1."""
    rng = np.random.default_rng(3)
    cache = {}
    amax = {}
    for i, name in enumerate(U.CONV_OUTPUTS):
        z = rng.normal(0.0, 1.0 + i, (2, 4, 4, 8))
        cache[name + ".z"] = z
        amax[name] = np.maximum(z, 0.0).max()
    cache["e1a.z"] = -np.abs(cache["e1a.z"])          # all zero after the ReLU
    s = U.activation_scales(cache)
    assert s[0] == 1.0
    for name, sc in zip(U.CONV_OUTPUTS[1:], s[1:]):
        assert amax[name] / sc == pytest.approx(448.0, rel=1e-12)
        assert U.e4m3_round(amax[name] / sc) == 448.0
