"""Pins of the per-pixel angular weights (oracle R9, the per-pixel form of
Sec. VI's weighting of each camera by its distance from the virtual one)
against an independent FP64 computation and the geometry."""
import math

import numpy as np
import pytest

import synthetic as S


def _fp64_weights(cams, view, Z, x, y, ks, unit=0.001):
    """Weights of cameras ks at view pixel (x, y) of depth Z (depth units),
    from the angle at the surface point (arccos in FP64), chord 2 sin(t/2)."""
    Pv = np.array([(x - view.cx) / view.fx * Z, (y - view.cy) / view.fy * Z, Z]) * unit
    P = view.R.T @ (Pv - view.t)                          # world point, metres
    Cv = -view.R.T @ view.t
    out = []
    for k in ks:
        Ck = -cams[k].R.T @ cams[k].t
        a, b = Ck - P, Cv - P
        th = math.acos(max(-1.0, min(1.0, float(a @ b) / (np.linalg.norm(a) * np.linalg.norm(b)))))
        out.append(1.0 / (2.0 * math.sin(th / 2.0) + 1e-3))
    return np.array(out)


def test_two_camera_weights_match_fp64(oracle_mod):
    """Two parallel cameras and the view between them: at every pixel both
    cameras see, the normalised top-2 weights equal the FP64 chord weights.
    Bound: the rays meet at ~0.03 rad, so 1 - cos ~ 4e-4 is formed from FP32
    values near 1 with an error of a few 1e-7, i.e. up to ~1e-3 relative in
    1 - cos, half that in the chord and the weight, and ~2.5e-4 in a share."""
    wl = S.workload("plain_2cam_320x240")
    cams, view = wl["cams"], wl["views"][0]
    out = oracle_mod.synthesize(cams, wl["rgb"], wl["depth"], view, wl["look_at"], pixel_weights=1,
                                crack_filter=0, hole_fill=0)
    both = (out["top3"][..., 1] > 0) & (out["hole"] == 0)
    assert both.mean() > 0.5
    ys, xs = np.nonzero(both)
    rng = np.random.default_rng(0)
    for i in rng.choice(len(ys), 300, replace=False):
        y, x = ys[i], xs[i]
        w = _fp64_weights(cams, view, float(out["depth"][y, x]), x, y, [0, 1])
        ref = np.sort(w / w.sum())[::-1]
        assert np.allclose(out["top3"][y, x, :2], ref, rtol=0, atol=2.5e-4)


def test_blend_share_follows_the_angles_at_the_point(oracle_mod):
    """Cameras at x = -50 mm and +50 mm, the view between them, a
    fronto-parallel plane at 1.5 m; camera 0 is black and camera 1 white, so
    an output channel is 255 x camera 1's weight share.  It follows the FP64
    chord weights pixel by pixel: left of centre the nearer camera 0 subtends
    the larger angle at the point and weighs less, right of centre the
    reverse, on the centre column they are equal.  With per-view weights
    every share is 1/2."""
    cams = S.rig_parallel(2, 160, 120, 150.0, 0.1)
    view = S.rig_parallel(1, 160, 120, 150.0, 0.1)[0]
    scene = S.scene_fronto_plane(1.5)
    rgb, dep = S.frames_for(scene, cams)
    rgb[0][...] = 0
    rgb[1][...] = 255
    O = np.array([0.0, 0.0, 1.5])
    out = oracle_mod.synthesize(cams, rgb, dep, view, O, pixel_weights=1, crack_filter=0, hole_fill=0)
    ok = out["top3"][..., 1] > 0
    ys, xs = np.nonzero(ok)
    for y, x in list(zip(ys, xs))[::97]:
        w = _fp64_weights(cams, view, float(out["depth"][y, x]), x, y, [0, 1])
        assert abs(int(out["rgb"][y, x, 0]) - 255.0 * w[1] / w.sum()) <= 0.51
    share = out["rgb"][60, :, 0].astype(int)
    cols = np.where(ok[60])[0]
    assert share[cols.min()] > 128 and share[cols.max()] < 128
    flat = oracle_mod.synthesize(cams, rgb, dep, view, O, crack_filter=0, hole_fill=0)
    assert np.all(np.abs(flat["rgb"][..., 0][ok].astype(int) - 128) <= 1)


def test_single_active_camera_is_unaffected(oracle_mod):
    """n_ref = 1 or a view on a camera: one contributor, so the per-pixel
    weights change nothing."""
    wl = S.workload("plain_9cam_1280x720", scale=0.2)
    for kw, v in ((dict(n_ref=1), wl["views"][30]), (dict(), wl["cams"][4].copy())):
        a = oracle_mod.synthesize(wl["cams"], wl["rgb"], wl["depth"], v, wl["look_at"], **kw)
        b = oracle_mod.synthesize(wl["cams"], wl["rgb"], wl["depth"], v, wl["look_at"], pixel_weights=1, **kw)
        assert np.array_equal(a["rgb"], b["rgb"]) and np.array_equal(a["keys"], b["keys"])


@pytest.mark.parametrize("fy_scale", [1.0, 1.3])
def test_weights_of_unequal_angles_match_fp64(oracle_mod, fy_scale):
    """The view 15 mm from camera 0 and 585 mm from camera 1 (both parallel,
    a fronto-parallel plane at 1.5 m): at the point the two rays meet camera
    0's at ~0.01 rad and camera 1's at ~0.4 rad, so the 1e-3 in
    w = 1 / (chord + 1e-3) weighs differently on the two and the shares pin
    the chord's absolute scale, sqrt(2 (1 - cos)) = 2 sin(t / 2), not only
    the ratio of the angles.  Bound as above: 1 - cos ~ 5e-5 for camera 0
    carries ~2e-3 relative FP32 error, ~1e-3 in its chord and weight, ~3e-5
    in camera 1's share of ~0.03.  The view's pixels are square or 1.3
    times taller than wide (fy = 1.3 fx), so x and y scale by their own
    focal lengths."""
    W, H, f = 160, 120, 150.0
    cams = [S.Camera(W, H, f, f, (W - 1) / 2, (H - 1) / 2, np.eye(3), -np.array([x, 0.0, 0.0]))
            for x in (0.0, 0.6)]
    view = S.Camera(W, H, f, f * fy_scale, (W - 1) / 2, (H - 1) / 2, np.eye(3), -np.array([0.015, 0.0, 0.0]))
    rgb, dep = S.frames_for(S.scene_fronto_plane(1.5), cams)
    out = oracle_mod.synthesize(cams, rgb, dep, view, [0.3, 0.0, 1.5], pixel_weights=1, crack_filter=0,
                                hole_fill=0)
    both = (out["top3"][..., 1] > 0) & (out["hole"] == 0)
    assert both.mean() > 0.3
    ys, xs = np.nonzero(both)
    for y, x in list(zip(ys, xs))[::53]:
        w = _fp64_weights(cams, view, float(out["depth"][y, x]), x, y, [0, 1])
        ref = np.sort(w / w.sum())[::-1]
        assert ref[1] < 0.05
        assert np.allclose(out["top3"][y, x, :2], ref, rtol=0, atol=1.5e-4)
