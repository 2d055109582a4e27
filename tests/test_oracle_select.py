"""Pins of the adaptive camera selection (oracle.select_cameras, Sec. V-C:
the N_Tx cameras closest to the virtual viewpoint are transmitted) and the
library's host implementation of it (no GPU)."""
import math

import numpy as np
import pytest

import synthetic as S


def _rig():
    """The 9-camera arc rig and its swing trajectory (tiny images: only the
    poses matter here)."""
    return {"cams": S.rig_arc(9, 90.0, 1.5, 64, 36, 50.0),
            "views": S.trajectory_arc(300, 22.5, 1.5, 64, 36, 50.0)}


def _arccos_nearest(cams, view, O, n):
    """Brute force with another formula for the angle: arccos of the
    normalised dot product."""
    cv = -(view.R.T @ view.t) - O
    th = []
    for c in cams:
        b = -(c.R.T @ c.t) - O
        th.append(math.acos(max(-1.0, min(1.0, float(cv @ b) / (np.linalg.norm(cv) * np.linalg.norm(b))))))
    return sorted(range(len(cams)), key=lambda k: (th[k], k))[:n]


def test_selection_matches_brute_force(oracle_mod):
    wl = _rig()
    O = np.zeros(3)
    for vi in (3, 47, 120, 201, 280):
        v = wl["views"][vi]
        for n in (1, 3, 5, 9):
            m = oracle_mod.select_cameras(wl["cams"], [v], O, n)
            assert m == sum(1 << k for k in _arccos_nearest(wl["cams"], v, O, n))
            assert bin(m).count("1") == n


def test_selection_invariants(oracle_mod):
    wl = _rig()
    cams, O = wl["cams"], np.zeros(3)
    # a view on a camera's pose selects that camera first
    for k in (0, 4, 8):
        assert oracle_mod.select_cameras(cams, [cams[k].copy()], O, 1) == 1 << k
    # nested in n_tx, all cameras at n_tx = K, union over views
    v1, v2 = wl["views"][0], wl["views"][75]
    prev = 0
    for n in range(1, 10):
        m = oracle_mod.select_cameras(cams, [v1], O, n)
        assert m & prev == prev
        prev = m
    assert prev == (1 << 9) - 1
    u = oracle_mod.select_cameras(cams, [v1, v2], O, 3)
    assert u == oracle_mod.select_cameras(cams, [v1], O, 3) | oracle_mod.select_cameras(cams, [v2], O, 3)
    # the camera symmetric to the view across the rig's middle swaps with it
    a = oracle_mod.select_cameras(cams, [S.arc_view(-20.0, 1.5, 64, 36, 50.0)], O, 3)
    b = oracle_mod.select_cameras(cams, [S.arc_view(20.0, 1.5, 64, 36, 50.0)], O, 3)
    assert a == int("".join(reversed(format(b, "09b"))), 2)


def test_library_selection_equals_oracle(oracle_mod):
    from fvv_helpers import lib
    F = lib()
    wl = _rig()
    r = F.rig(wl["cams"], [0, 0, 0])
    views = [wl["views"][i] for i in (5, 60, 150, 222)]
    for n in (1, 3, 5, 9):
        for vs in ([views[0]], views[1:3], views):
            assert F.fvv_select_cameras(r, vs, n) == oracle_mod.select_cameras(wl["cams"], vs, np.zeros(3), n)
    with pytest.raises(F.FvvError):
        F.fvv_select_cameras(r, views, 0)
    with pytest.raises(F.FvvError):
        F.fvv_select_cameras(r, views, 10)


def test_ties_go_to_the_lower_camera(oracle_mod):
    """A view exactly midway between two cameras of a mirror-symmetric pair
    (angles equal to the last bit): one camera to send is the lower index,
    two are both; the same with the pair's indices swapped."""
    cams = S.rig_parallel(2, 64, 36, 50.0, 0.2)
    O = np.array([0.0, 0.0, 1.5])
    view = S.rig_parallel(1, 64, 36, 50.0, 0.2)[0]
    assert oracle_mod.select_cameras(cams, [view], O, 1) == 0b01
    assert oracle_mod.select_cameras(cams, [view], O, 2) == 0b11
    assert oracle_mod.select_cameras(cams[::-1], [view], O, 1) == 0b01
    # the library's host selection takes the same tie rule
    from fvv_helpers import lib
    F = lib()
    for cs in (cams, cams[::-1]):
        assert F.fvv_select_cameras(F.rig(cs, O), [view], 1) == 0b01


def test_selection_is_invariant_to_moving_the_whole_rig(oracle_mod):
    """Closeness is the angle about the rig's look-at point, so translating
    the cameras, the views and that point together changes no selection
    (the rig's centre is not the world origin in general)."""
    wl = _rig()
    off = np.array([1.0, -2.0, 3.0])

    def moved(c):
        m = c.copy()
        m.t = c.t - c.R @ off                 # centre C + off
        return m
    cams = [moved(c) for c in wl["cams"]]
    for vi in (10, 90, 170, 250):
        v = wl["views"][vi]
        for n in (1, 3, 5):
            assert (oracle_mod.select_cameras(cams, [moved(v)], off, n) ==
                    oracle_mod.select_cameras(wl["cams"], [v], np.zeros(3), n))
    from fvv_helpers import lib
    F = lib()
    r = F.rig(cams, off)
    vs = [moved(wl["views"][i]) for i in (10, 90)]
    assert F.fvv_select_cameras(r, vs, 3) == oracle_mod.select_cameras(cams, vs, off, 3)
