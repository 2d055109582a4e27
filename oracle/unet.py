"""FP64 CPU oracle of the refinement network (forward, backward, loss, Adam).

TEST INFRASTRUCTURE ONLY (tests, smoke check, benchmark CPU leg).  The paper
has no learned stage; the network is the one the refinement target
specifies: a 3-level U-Net with 3x3 convolutions (pad 1) and ReLU,
32/64/128 channels, 8 input channels (RGB / 255, depth / z_far, hole mask,
the 3 largest blend weights) and 3 output channels added to the blended RGB.

Readings (the target leaves them open): two convolutions per level, 2x2 max
pooling down, nearest-neighbour 2x upsampling, skip connections by channel
concatenation (decoder input = [upsampled, encoder]), a final 1x1
convolution, output = clamp(rgb + residual, 0, 1), mean-squared-error loss.

Layout: activations NHWC; a 3x3 weight is W[co, ky, kx, ci] (the reduction
index (ky, kx, ci) is contiguous); a 1x1 weight is W[co, ci].
Plain numpy: every step is its definition written out with tensordot.
"""
from __future__ import annotations

import numpy as np

LAYERS_3x3 = ["e1a", "e1b", "e2a", "e2b", "ba", "bb", "d2a", "d2b", "d1a", "d1b"]


def layer_shapes(widths=(32, 64, 128), c_in=8, c_out=3):
    w1, w2, w3 = widths
    return {
        "e1a": (w1, c_in), "e1b": (w1, w1),
        "e2a": (w2, w1), "e2b": (w2, w2),
        "ba": (w3, w2), "bb": (w3, w3),
        "d2a": (w2, w3 + w2), "d2b": (w2, w2),
        "d1a": (w1, w2 + w1), "d1b": (w1, w1),
        "out": (c_out, w1),
    }


def init_params(widths=(32, 64, 128), seed=0, c_in=8, c_out=3, out_scale=0.1):
    """He-normal 3x3 weights, zero biases, a small final 1x1 layer."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, (co, ci) in layer_shapes(widths, c_in, c_out).items():
        if name == "out":
            p[name + ".w"] = rng.standard_normal((co, ci)) * out_scale * np.sqrt(1.0 / ci)
        else:
            p[name + ".w"] = rng.standard_normal((co, 3, 3, ci)) * np.sqrt(2.0 / (9 * ci))
        p[name + ".b"] = np.zeros(co)
    return p


# ---------------------------------------------------------------------------
# primitives (forward / backward by definition)
# ---------------------------------------------------------------------------

def conv3x3(x, w, b):
    """y[n, y, x, co] = b[co] + sum_{ky,kx,ci} w[co,ky,kx,ci] xp[n, y+ky, x+kx, ci],
    xp = x zero-padded by one pixel."""
    n, h, wd, ci = x.shape
    xp = np.zeros((n, h + 2, wd + 2, ci))
    xp[:, 1:-1, 1:-1] = x
    y = np.zeros((n, h, wd, w.shape[0])) + b
    for ky in range(3):
        for kx in range(3):
            y += np.tensordot(xp[:, ky:ky + h, kx:kx + wd, :], w[:, ky, kx, :], axes=([3], [1]))
    return y


def conv3x3_backward(x, w, dy):
    """Gradients of conv3x3 with respect to x, w and b."""
    n, h, wd, ci = x.shape
    xp = np.zeros((n, h + 2, wd + 2, ci))
    xp[:, 1:-1, 1:-1] = x
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w)
    for ky in range(3):
        for kx in range(3):
            dxp[:, ky:ky + h, kx:kx + wd, :] += np.tensordot(dy, w[:, ky, kx, :], axes=([3], [0]))
            dw[:, ky, kx, :] = np.tensordot(dy, xp[:, ky:ky + h, kx:kx + wd, :],
                                            axes=([0, 1, 2], [0, 1, 2]))
    return dxp[:, 1:-1, 1:-1], dw, dy.sum(axis=(0, 1, 2))


def conv1x1(x, w, b):
    return np.tensordot(x, w, axes=([3], [1])) + b


def conv1x1_backward(x, w, dy):
    return (np.tensordot(dy, w, axes=([3], [0])),
            np.tensordot(dy, x, axes=([0, 1, 2], [0, 1, 2])),
            dy.sum(axis=(0, 1, 2)))


def relu(x):
    return np.maximum(x, 0.0)


def relu_backward(x, dy):
    return dy * (x > 0)


def maxpool2(x):
    """2x2 max pooling, stride 2 (H and W even).  Returns (y, argmax index
    0..3 in the order (0,0), (0,1), (1,0), (1,1); the first maximum wins)."""
    n, h, wd, c = x.shape
    q = np.stack([x[:, 0::2, 0::2], x[:, 0::2, 1::2], x[:, 1::2, 0::2], x[:, 1::2, 1::2]], axis=0)
    return q.max(axis=0), q.argmax(axis=0)


def maxpool2_backward(arg, dy):
    n, h2, w2, c = dy.shape
    dx = np.zeros((n, 2 * h2, 2 * w2, c))
    for i, (oy, ox) in enumerate(((0, 0), (0, 1), (1, 0), (1, 1))):
        dx[:, oy::2, ox::2] = dy * (arg == i)
    return dx


def up2(x):
    return x.repeat(2, axis=1).repeat(2, axis=2)


def up2_backward(dy):
    return dy[:, 0::2, 0::2] + dy[:, 0::2, 1::2] + dy[:, 1::2, 0::2] + dy[:, 1::2, 1::2]


# ---------------------------------------------------------------------------
# network
# ---------------------------------------------------------------------------

def forward(p, x, rgb):
    """x: (N, H, W, 8) input features; rgb: (N, H, W, 3) blended colour in
    [0, 1].  Returns (pred, cache); pred = clamp(rgb + residual, 0, 1)."""
    c = {"x": x, "rgb": rgb}

    def cr(name, inp):
        z = conv3x3(inp, p[name + ".w"], p[name + ".b"])
        c[name + ".in"], c[name + ".z"] = inp, z
        return relu(z)

    e1 = cr("e1b", cr("e1a", x))
    p1, c["p1.arg"] = maxpool2(e1)
    e2 = cr("e2b", cr("e2a", p1))
    p2, c["p2.arg"] = maxpool2(e2)
    bt = cr("bb", cr("ba", p2))
    u2 = up2(bt)
    d2 = cr("d2b", cr("d2a", np.concatenate([u2, e2], axis=3)))
    u1 = up2(d2)
    d1 = cr("d1b", cr("d1a", np.concatenate([u1, e1], axis=3)))
    res = conv1x1(d1, p["out.w"], p["out.b"])
    s = rgb + res
    c["d1"], c["s"], c["widths"] = d1, s, (e1.shape[3], e2.shape[3], bt.shape[3])
    return np.clip(s, 0.0, 1.0), c


def backward(p, c, dpred):
    """Gradients of every parameter given dL/dpred."""
    g = {}
    s = c["s"]
    ds = dpred * ((s > 0.0) & (s < 1.0))

    def crb(name, dy_relu):
        dz = relu_backward(c[name + ".z"], dy_relu)
        dx, g[name + ".w"], g[name + ".b"] = conv3x3_backward(c[name + ".in"], p[name + ".w"], dz)
        return dx

    dd1, g["out.w"], g["out.b"] = conv1x1_backward(c["d1"], p["out.w"], ds)
    w1, w2, w3 = c["widths"]
    dcat1 = crb("d1a", crb("d1b", dd1))
    du1, de1_skip = dcat1[..., :w2], dcat1[..., w2:]
    dd2 = up2_backward(du1)
    dcat2 = crb("d2a", crb("d2b", dd2))
    du2, de2_skip = dcat2[..., :w3], dcat2[..., w3:]
    dbt = up2_backward(du2)
    dp2 = crb("ba", crb("bb", dbt))
    de2 = maxpool2_backward(c["p2.arg"], dp2) + de2_skip
    dp1 = crb("e2a", crb("e2b", de2))
    de1 = maxpool2_backward(c["p1.arg"], dp1) + de1_skip
    crb("e1a", crb("e1b", de1))
    return g


def mse(pred, target):
    """Mean squared error over every element; returns (loss, dL/dpred)."""
    d = pred - target
    return float(np.mean(d * d)), 2.0 * d / d.size


def adam_step(p, g, state, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (bias-corrected), in place on p."""
    t = state.get("t", 0) + 1
    state["t"] = t
    for k in p:
        m = state.setdefault("m." + k, np.zeros_like(p[k]))
        v = state.setdefault("v." + k, np.zeros_like(p[k]))
        m[...] = b1 * m + (1 - b1) * g[k]
        v[...] = b2 * v + (1 - b2) * g[k] * g[k]
        mh = m / (1 - b1 ** t)
        vh = v / (1 - b2 ** t)
        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)


def features(rgb8, depth, hole, top3, z_far):
    """The 8 input channels from a plain synthesis: RGB / 255, depth / z_far,
    hole mask (0/1), three largest normalised blend weights."""
    return np.concatenate([rgb8.astype(np.float64) / 255.0,
                           (depth.astype(np.float64) / z_far)[..., None],
                           hole.astype(np.float64)[..., None],
                           top3.astype(np.float64)], axis=-1)


# ---------------------------------------------------------------------------
# FP8 form: OCP E4M3 (1 sign bit, 4 exponent bits with bias 7, 3 mantissa
# bits; normal numbers 2^(e-7) (1 + m/8) for e = 1..15, except e = 15, m = 7
# which is NaN, so the largest finite value is 448; subnormals (m/8) 2^-6;
# no infinities).  Conversions round to nearest, ties to even mantissa, and
# saturate to +-448.
# ---------------------------------------------------------------------------
E4M3_MAX = 448.0


def e4m3_round(x):
    """The E4M3 value nearest to x (ties to even), saturated to [-448, 448]."""
    x = np.asarray(x, np.float64)
    a = np.abs(x)
    _, ex = np.frexp(a)                       # a = f 2^ex with f in [0.5, 1): binade 2^(ex-1)
    e = np.clip(ex - 1, -6, 8)                # below 2^-6 the spacing stays 2^-9 (subnormals)
    step = np.ldexp(1.0, e - 3)               # 3 mantissa bits
    q = np.minimum(np.round(a / step) * step, E4M3_MAX)   # np.round: half to even
    return np.where(np.signbit(x), -q, q)


def e4m3_encode(q):
    """Bytes of E4M3-representable values (as returned by e4m3_round)."""
    q = np.asarray(q, np.float64)
    a = np.abs(q)
    sign = np.signbit(q).astype(np.uint8)
    _, ex = np.frexp(a)
    e = ex - 1
    sub = a < 2.0 ** -6
    E = np.where(sub, 0, e + 7)
    M = np.where(sub, a / 2.0 ** -9, (np.ldexp(a, -np.where(sub, 0, e)) - 1.0) * 8.0)
    return ((sign << 7) | (E.astype(np.uint8) << 3) | M.astype(np.uint8)).astype(np.uint8)


def e4m3_decode(b):
    """Values of E4M3 bytes (the NaN codes 0x7f / 0xff decode to NaN)."""
    b = np.asarray(b, np.uint8).astype(np.int64)
    s = np.where(b >> 7, -1.0, 1.0)
    E = (b >> 3) & 15
    M = b & 7
    v = np.where(E == 0, M / 8.0 * 2.0 ** -6, (1.0 + M / 8.0) * np.ldexp(1.0, E - 7))
    v = np.where((E == 15) & (M == 7), np.nan, v)
    return s * v


# ---------------------------------------------------------------------------
# FP8 inference form of the network (post-training quantisation)
# ---------------------------------------------------------------------------
CONV_OUTPUTS = ["e1a", "e1b", "e2a", "e2b", "ba", "bb", "d2a", "d2b", "d1a", "d1b"]


def activation_scales(cache):
    """Per-tensor scales amax / 448 of the ten conv outputs of a forward pass
    (ReLU outputs; a tensor that is all zero gets scale 1)."""
    out = []
    for name in CONV_OUTPUTS:
        a = np.abs(relu(cache[name + ".z"])).max()
        out.append(a / E4M3_MAX if a > 0 else 1.0)
    return np.array(out)


def forward_e4m3(p, x, rgb, act_scales, s0=2.0 ** -8):
    """The network with every activation stored as E4M3 codes of one
    per-tensor scale: the input features at s0, conv output t at
    act_scales[t].  Layer l with input parts (codes X_j, scale s_j) takes
    weights W' = W s_j / s_1 on part j's channels, one weight scale
    s_w = max|W'| / 448 and codes Q = e4m3(W' / s_w); its output codes are
    e4m3(relu(s_1 s_w conv(X, Q) + b) / s_out).  Max pooling and upsampling
    move codes; the head uses the dequantised last activation.
    Returns the clamped prediction."""
    S = dict(zip(CONV_OUTPUTS, act_scales))

    def layer(name, parts, s_out):
        xq = np.concatenate([c for c, _ in parts], axis=3)
        f = np.concatenate([np.full(c.shape[3], s / parts[0][1]) for c, s in parts])
        wp = p[name + ".w"] * f
        s_w = np.abs(wp).max() / E4M3_MAX
        s_w = s_w if s_w > 0 else 1.0
        acc = conv3x3(xq, e4m3_round(wp / s_w), np.zeros(wp.shape[0]))
        return e4m3_round(relu(acc * (parts[0][1] * s_w) + p[name + ".b"]) / s_out)

    X0 = e4m3_round(x / s0)
    e1a = layer("e1a", [(X0, s0)], S["e1a"])
    e1 = layer("e1b", [(e1a, S["e1a"])], S["e1b"])
    p1, _ = maxpool2(e1)
    e2a = layer("e2a", [(p1, S["e1b"])], S["e2a"])
    e2 = layer("e2b", [(e2a, S["e2a"])], S["e2b"])
    p2, _ = maxpool2(e2)
    ba = layer("ba", [(p2, S["e2b"])], S["ba"])
    bt = layer("bb", [(ba, S["ba"])], S["bb"])
    d2a = layer("d2a", [(up2(bt), S["bb"]), (e2, S["e2b"])], S["d2a"])
    d2 = layer("d2b", [(d2a, S["d2a"])], S["d2b"])
    d1a = layer("d1a", [(up2(d2), S["d2b"]), (e1, S["e1b"])], S["d1a"])
    d1 = layer("d1b", [(d1a, S["d1a"])], S["d1b"])
    res = conv1x1(d1 * S["d1b"], p["out.w"], p["out.b"])
    return np.clip(rgb + res, 0.0, 1.0)
