"""Pins of the oracle's warp (steps a, b): the DIBR geometry of Sec. VI.

Each test compares the oracle with something other than itself: the
identity pose, the closed-form shift f B / Z of a fronto-parallel plane,
an independent FP64 world-point projection, and a brute force over
single-point splats.
"""
import math
import os

import numpy as np
import pytest

import synthetic as S

HERE = os.path.dirname(os.path.abspath(__file__))


def _cam(width, height, f, center, R=None, fy=None, cx=None, cy=None):
    R = np.eye(3) if R is None else np.asarray(R, float)
    c = np.asarray(center, float)
    return S.Camera(width, height, f, f if fy is None else fy,
                    (width - 1) / 2.0 if cx is None else cx,
                    (height - 1) / 2.0 if cy is None else cy, R, -R @ c)


def _project_fp64(cam_src, cam_dst, u, v, z_mm):
    """Independent FP64 geometry: source pixel + depth -> world -> target."""
    x = np.stack([(u - cam_src.cx) / cam_src.fx * z_mm / 1000.0,
                  (v - cam_src.cy) / cam_src.fy * z_mm / 1000.0,
                  z_mm / 1000.0], axis=-1)
    P = (x - cam_src.t) @ cam_src.R           # R.T @ (x - t)
    q = P @ cam_dst.R.T + cam_dst.t
    ud = cam_dst.fx * q[:, 0] / q[:, 2] + cam_dst.cx
    vd = cam_dst.fy * q[:, 1] / q[:, 2] + cam_dst.cy
    return ud, vd, q[:, 2] * 1000.0


def test_identity_pose_reproduces_input(oracle_mod):
    """A virtual camera placed on a reference camera reproduces its frame:
    every pixel with depth maps onto itself, pixels without depth are holes."""
    for name, k, scale in (("plain_2cam_320x240", 0, 1.0), ("plain_9cam_1280x720", 4, 0.25)):
        wl = S.workload(name, scale=scale)
        view = wl["cams"][k].copy()
        out = oracle_mod.synthesize(wl["cams"], wl["rgb"], wl["depth"], view, wl["look_at"],
                                    crack_filter=0, hole_fill=0)
        valid = wl["depth"][k] > 0
        assert np.array_equal(out["rgb"][valid], wl["rgb"][k][valid])
        assert np.array_equal(out["hole"].astype(bool), ~valid)
        assert np.allclose(out["depth"][valid], wl["depth"][k][valid].astype(np.float32),
                           rtol=1e-6, atol=0)
        z, cam, src = oracle_mod.key_fields(out["keys"])
        yy, xx = np.nonzero(valid)
        assert np.all(cam[valid] == k)
        assert np.array_equal(src[valid], yy * view.width + xx)


def test_identity_pose_with_filter_on_plane(oracle_mod):
    """With the crack filter on, a sliver-free scene (one textured plane)
    still reproduces the input exactly."""
    cams = S.rig_parallel(2, 96, 64, 120.0, 0.1)
    rgb, dep = S.frames_for(S.scene_fronto_plane(1.5), cams)
    out = oracle_mod.synthesize(cams, rgb, dep, cams[1].copy(), [0, 0, 1.5])
    assert np.array_equal(out["rgb"], rgb[1])
    assert not out["hole"].any()


def _golden_shifts():
    rows = []
    with open(os.path.join(HERE, "golden", "fronto_plane_shifts.txt")) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                f, b, z, sh, frac = (float(x) for x in line.split())
                rows.append((f, b, z, sh, frac))
    return rows


@pytest.mark.parametrize("row", _golden_shifts())
@pytest.mark.parametrize("axis", ["x", "y"])
def test_fronto_plane_shift(oracle_mod, row, axis):
    """A fronto-parallel plane at Z shifts by f B / Z between parallel cameras;
    an exact .5 shift rounds up (floor(u' + 0.5))."""
    f, b_mm, z_mm, shift, frac = row
    W, H = 320, 240
    B = b_mm / 1000.0
    e = np.array([1.0, 0.0, 0.0]) if axis == "x" else np.array([0.0, 1.0, 0.0])
    cam0 = _cam(W, H, f, -0.5 * B * e)
    cam1 = _cam(W, H, f, 0.5 * B * e)
    view = _cam(W, H, f, (-0.5 + frac) * B * e)
    assert math.isclose(f * frac * b_mm / z_mm, shift, rel_tol=1e-12)
    dep = np.full((H, W), int(z_mm), np.uint16)
    M, N, _ = oracle_mod.compose([cam0, cam1], view, [0, 0, z_mm / 1000.0])
    keys = oracle_mod.warp_splat([cam0], [dep], M[:1], np.ones(1, np.float32), W, H,
                                 oracle_mod.options())
    z, cam, src = oracle_mod.key_fields(keys)
    su, sv = src % W, src // W
    xx, yy = np.meshgrid(np.arange(W), np.arange(H))
    # the view sits frac*B towards +axis from cam0: content moves by -shift
    s_along, d_along, n_along = (su, xx, W) if axis == "x" else (sv, yy, H)
    s_other, d_other = (sv, yy) if axis == "x" else (su, xx)
    # FP64 reference: the first source index whose rounded target is this pixel
    tgt = np.floor(np.arange(n_along) - shift + 0.5).astype(int)
    first = {}
    for s_i, t_i in enumerate(tgt):
        if 0 <= t_i < n_along and t_i not in first:
            first[t_i] = s_i
    exp = np.array([first.get(i, -1) for i in range(n_along)])
    exp_map = exp[d_along]
    filled = exp_map >= 0
    assert np.array_equal(cam[filled], np.zeros(filled.sum(), int))
    assert np.array_equal(s_along[filled], exp_map[filled])
    assert np.array_equal(s_other[filled], d_other[filled])
    assert np.all(z[filled] == np.float32(z_mm))
    assert np.all(src[~filled] == -1)
    if shift == 7.5:
        assert exp[0] == 7          # tie at .5 rounds up: u - 7.5 -> u - 7


def test_zoom_intrinsics(oracle_mod):
    """Same pose, different intrinsics: u' = fx_v (u - cx) / fx + cx_v."""
    W, H = 64, 48
    src = _cam(W, H, 80.0, [0, 0, 0])
    view = _cam(W, H, 100.0, [0, 0, 0], fy=90.0, cx=30.25, cy=20.5)
    rng = np.random.default_rng(3)
    dep = np.zeros((H, W), np.uint16)
    sel = rng.choice(W * H, 40, replace=False)
    dep.ravel()[sel] = rng.integers(500, 6000, sel.size)
    M, _, _ = oracle_mod.compose([src], view, [0, 0, 1])
    keys = oracle_mod.warp_splat([src], [dep], M, np.ones(1, np.float32), W, H)
    z, cam, s = oracle_mod.key_fields(keys)
    got = {int(si): (x, y, zz) for (y, x), si, zz in zip(np.argwhere(s >= 0), s[s >= 0], z[s >= 0])}
    for si in sel:
        u, v = si % W, si // W
        ue = 100.0 * (u - src.cx) / 80.0 + 30.25
        ve = 90.0 * (v - src.cy) / 80.0 + 20.5
        tu, tv = math.floor(ue + 0.5), math.floor(ve + 0.5)
        inside = 0 <= tu < W and 0 <= tv < H
        if inside:
            assert int(si) in got or any(  # may lose to a nearer point on the same pixel
                zz < dep.ravel()[si] for (x, y, zz) in got.values() if (x, y) == (tu, tv))
            if int(si) in got:
                x, y, zz = got[int(si)]
                assert (x, y) == (tu, tv)
                assert zz == np.float32(dep.ravel()[si])
        else:
            assert int(si) not in got


@pytest.mark.parametrize("seed,fy_scale", [(0, 1.0), (1, 1.0), (2, 1.0), (3, 1.2)])
def test_general_pose_matches_fp64_projection(oracle_mod, seed, fy_scale):
    """Arbitrary poses on the nine-camera arc: each splatted sparse source
    point lands on the pixel an independent FP64 projection predicts (away
    from rounding ties) with its target-camera depth.  The last case gives
    the source cameras pixels 1.2 times taller than wide (fy = 1.2 fx)."""
    rng = np.random.default_rng(seed)
    W, H, f = 160, 90, 125.0
    cams = S.rig_arc(9, 90.0, 1.5, W, H, f)
    for c in cams:
        c.fy = c.fx * fy_scale
    view = S.arc_view(rng.uniform(-40, 40), 1.5 + rng.uniform(-0.3, 0.3), W, H,
                      f * rng.uniform(0.8, 1.25))
    M, N, _ = oracle_mod.compose(cams, view, [0, 0, 0])
    for k in range(9):
        dep = np.zeros((H, W), np.uint16)
        sel = rng.choice(W * H, 25, replace=False)
        dep.ravel()[sel] = rng.integers(900, 2500, sel.size)
        w = np.zeros(9, np.float32)
        w[k] = 1.0
        keys = oracle_mod.warp_splat(cams, [dep if i == k else np.zeros_like(dep) for i in range(9)],
                                     M, w, W, H)
        z, cam, s = oracle_mod.key_fields(keys)
        hits = {int(si): (int(x), int(y), float(zz))
                for (y, x), si, zz in zip(np.argwhere(s >= 0), s[s >= 0], z[s >= 0])}
        u = (sel % W).astype(float)
        v = (sel // W).astype(float)
        ud, vd, zd = _project_fp64(cams[k], view, u, v, dep.ravel()[sel].astype(float))
        checked = 0
        for i, si in enumerate(sel):
            if abs((ud[i] + 0.5) % 1.0) < 1e-3 or abs((vd[i] + 0.5) % 1.0) < 1e-3:
                continue
            tu, tv = math.floor(ud[i] + 0.5), math.floor(vd[i] + 0.5)
            if not (0 <= tu < W and 0 <= tv < H) or zd[i] <= 1.0:
                assert int(si) not in hits
                continue
            if int(si) in hits:
                x, y, zz = hits[int(si)]
                assert (x, y) == (tu, tv)
                assert abs(zz - zd[i]) <= 1e-5 * zd[i]
                checked += 1
        assert checked >= 5


@pytest.mark.parametrize("seed", [0, 1])
def test_backward_map_matches_fp64(oracle_mod, seed):
    """The backward map N_k takes (x Z, y Z, Z, 1) of the view to camera k's
    pixel and depth, as an independent FP64 projection does."""
    rng = np.random.default_rng(10 + seed)
    W, H, f = 200, 120, 160.0
    cams = S.rig_arc(5, 60.0, 2.0, W, H, f)
    view = S.arc_view(rng.uniform(-30, 30), 2.2, W, H, 150.0)
    M, N, _ = oracle_mod.compose(cams, view, [0, 0, 0])
    x = rng.uniform(0, W - 1, 50)
    y = rng.uniform(0, H - 1, 50)
    Z = rng.uniform(1000, 3000, 50)
    for k in range(5):
        ue, ve, ze = _project_fp64(view, cams[k], x, y, Z)
        n = N[k].astype(np.float64)
        h = n[:, :3] @ np.stack([x * Z, y * Z, Z]) + n[:, 3:4]
        assert np.allclose(h[0] / h[2], ue, atol=2e-3)
        assert np.allclose(h[1] / h[2], ve, atol=2e-3)
        assert np.allclose(h[2], ze, rtol=1e-6)
        m = M[k].astype(np.float64)
        uk, vk, zk = _project_fp64(cams[k], view, x, y, Z)
        h2 = m[:, :3] @ np.stack([x * Z, y * Z, Z]) + m[:, 3:4]
        assert np.allclose(h2[0] / h2[2], uk, atol=2e-3)
        assert np.allclose(h2[2], zk, rtol=1e-6)


def _splat_single(oracle_mod, cams, deps, M, w, Wv, Hv, k, v, u):
    single = [np.zeros_like(d) for d in deps]
    single[k][v, u] = deps[k][v, u]
    keys = oracle_mod.warp_splat(cams, single, M, w, Wv, Hv)
    nz = np.argwhere(keys != oracle_mod.KEY_EMPTY)
    assert len(nz) <= 1
    return None if len(nz) == 0 else (tuple(nz[0]), keys[tuple(nz[0])])


@pytest.mark.parametrize("case", ["random", "ties"])
def test_zbuffer_matches_brute_force(oracle_mod, case):
    """Tiny images: the z-buffer equals the per-pixel minimum over every
    source point splatted alone; each key carries its camera and source
    index; equal depths resolve by camera, then source index."""
    rng = np.random.default_rng(7)
    Wv, Hv, W, H = 8, 6, 8, 6
    if case == "random":
        cams = [_cam(W, H, 6.0, [x, y, 0.0]) for x, y in ((-0.1, 0.0), (0.05, 0.02), (0.12, -0.03))]
        view = _cam(Wv, Hv, 7.0, [0.02, 0.01, 0.05])
        deps = [rng.integers(400, 1200, (H, W)).astype(np.uint16) for _ in cams]
        for d in deps:
            d[rng.random((H, W)) < 0.2] = 0
    else:
        cams = [_cam(W, H, 6.0, [0, 0, 0]) for _ in range(3)]
        view = _cam(Wv, Hv, 3.0, [0, 0, 0])         # minification: many-to-one
        deps = [np.full((H, W), 1000, np.uint16) for _ in cams]
    M, _, _ = oracle_mod.compose(cams, view, [0, 0, 1.0])
    w = np.ones(3, np.float32)
    full = oracle_mod.warp_splat(cams, deps, M, w, Wv, Hv)
    brute = np.full((Hv, Wv), oracle_mod.KEY_EMPTY, np.uint64)
    n_hit = 0
    for k in range(3):
        for v in range(H):
            for u in range(W):
                if deps[k][v, u] == 0:
                    continue
                r = _splat_single(oracle_mod, cams, deps, M, w, Wv, Hv, k, v, u)
                if r is None:
                    continue
                n_hit += 1
                pos, key = r
                z, cam, src = oracle_mod.key_fields(np.array([key]))
                assert cam[0] == k and src[0] == v * W + u
                brute[pos] = min(brute[pos], key)
    assert n_hit > 20
    assert np.array_equal(full, brute)
    if case == "ties":
        z, cam, src = oracle_mod.key_fields(full)
        assert np.all(cam[full != oracle_mod.KEY_EMPTY] == 0)
