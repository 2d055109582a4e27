"""Analytic scenes, rigs and trajectories, ray-cast in FP64.

Conventions (shared by every consumer of these frames):
  * world and camera axes: x right, y down, z forward;
  * a camera maps world -> camera by ``x_cam = R @ X + t`` (metres);
  * pixel (u, v) has its centre at integer (u, v); the ray through it is
    ``R.T @ ((u - cx) / fx, (v - cy) / fy, 1)``, so the ray parameter of a hit
    is the camera-space depth z;
  * depth frames are uint16 millimetres of camera-space z, 0 = no depth;
    in layered frames 65535 (``DEPTH_BG``) marks a background pixel, whose
    depth is not sent (a separate static background model holds it).

The rig shapes follow the paper's test set-up (Sec. IX: nine cameras on an
arc; swing / still trajectories); the scenes stand in for its captured
sequences, which are not available.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np

_EPS_T = 1e-6
DEPTH_BG = 65535


@dataclass
class Camera:
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    R: np.ndarray          # (3, 3) world -> camera rotation
    t: np.ndarray          # (3,) world -> camera translation, metres

    @property
    def center(self) -> np.ndarray:
        return -self.R.T @ self.t

    def copy(self) -> "Camera":
        return Camera(self.width, self.height, self.fx, self.fy, self.cx, self.cy,
                      self.R.copy(), self.t.copy())


def look_at_camera(center, target, width: int, height: int, f: float,
                   down=(0.0, 1.0, 0.0)) -> Camera:
    """Pinhole camera at ``center`` looking at ``target`` (world y points down)."""
    c = np.asarray(center, dtype=np.float64)
    z = np.asarray(target, dtype=np.float64) - c
    z = z / np.linalg.norm(z)
    x = np.cross(np.asarray(down, dtype=np.float64), z)
    x = x / np.linalg.norm(x)
    y = np.cross(z, x)
    R = np.stack([x, y, z])
    t = -R @ c
    return Camera(int(width), int(height), float(f), float(f),
                  (width - 1) / 2.0, (height - 1) / 2.0, R, t)


# --------------------------------------------------------------------------
# scene primitives
# --------------------------------------------------------------------------

@dataclass
class Sphere:
    center: np.ndarray
    radius: float
    albedo: np.ndarray            # RGB in [0, 255]


@dataclass
class Box:
    center: np.ndarray
    half: np.ndarray              # half extents (x, y, z) in the box frame
    yaw: float                    # rotation about the world y axis, radians
    albedo: np.ndarray


@dataclass
class Plane:
    point: np.ndarray
    normal: np.ndarray            # unit normal
    color_a: np.ndarray
    color_b: np.ndarray
    square: float                 # checker square size, metres (0 = plain colour_a)
    u_axis: np.ndarray = field(default_factory=lambda: np.array([1.0, 0.0, 0.0]))
    v_axis: np.ndarray = field(default_factory=lambda: np.array([0.0, 1.0, 0.0]))


@dataclass
class CylinderWall:
    """Vertical cylinder (axis parallel to y through ``center``), seen from inside."""
    center: np.ndarray
    radius: float
    color_a: np.ndarray
    color_b: np.ndarray
    cell: float                   # checker cell size along the wall, metres


@dataclass
class Scene:
    spheres: List[Sphere] = field(default_factory=list)
    boxes: List[Box] = field(default_factory=list)
    planes: List[Plane] = field(default_factory=list)
    walls: List[CylinderWall] = field(default_factory=list)
    light_to: np.ndarray = field(
        default_factory=lambda: np.array([-1.0, -1.0, -2.0]) / math.sqrt(6.0))
    ambient: float = 0.2


# --------------------------------------------------------------------------
# ray casting
# --------------------------------------------------------------------------

def _rays(cam: Camera):
    u = np.arange(cam.width, dtype=np.float64)
    v = np.arange(cam.height, dtype=np.float64)
    uu, vv = np.meshgrid(u, v)
    dc = np.stack([(uu - cam.cx) / cam.fx, (vv - cam.cy) / cam.fy,
                   np.ones_like(uu)], axis=-1)
    dw = dc @ cam.R                   # row vectors: R.T @ d  ==  d @ R
    return dw.reshape(-1, 3)


def _bbox_pixels(cam: Camera, center, radius):
    """Conservative pixel rectangle that contains the image of a ball."""
    corners = np.array([[sx, sy, sz] for sx in (-1, 1) for sy in (-1, 1)
                        for sz in (-1, 1)], dtype=np.float64) * radius + center
    pc = corners @ cam.R.T + cam.t
    if np.any(pc[:, 2] <= 1e-3):
        return 0, cam.width, 0, cam.height
    u = cam.fx * pc[:, 0] / pc[:, 2] + cam.cx
    v = cam.fy * pc[:, 1] / pc[:, 2] + cam.cy
    u0 = max(0, int(math.floor(u.min())) - 1)
    u1 = min(cam.width, int(math.ceil(u.max())) + 2)
    v0 = max(0, int(math.floor(v.min())) - 1)
    v1 = min(cam.height, int(math.ceil(v.max())) + 2)
    if u0 >= u1 or v0 >= v1:
        return None
    return u0, u1, v0, v1


def render(scene: Scene, cam: Camera):
    """Ray-cast ``scene`` from ``cam`` in FP64.

    Returns dict with ``rgb`` (H, W, 3) float64 in [0, 255] before rounding,
    ``z`` (H, W) camera-space depth in metres (inf = no hit), ``obj`` (H, W)
    int32 object id (-1 = no hit), ``normal`` (H, W, 3) and ``point`` (H, W, 3).
    """
    H, W = cam.height, cam.width
    n = H * W
    d = _rays(cam)
    C = cam.center
    tbest = np.full(n, np.inf)
    obj = np.full(n, -1, dtype=np.int32)
    nrm = np.zeros((n, 3))
    alb = np.zeros((n, 3))
    oid = 0
    pix = np.arange(n).reshape(H, W)

    def take(idx, t, normal, albedo, ident):
        better = t < tbest[idx]
        if not np.any(better):
            return
        j = idx[better]
        tbest[j] = t[better]
        obj[j] = ident
        nrm[j] = normal[better]
        alb[j] = albedo[better] if albedo.ndim == 2 else albedo

    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        for w in scene.walls:
            idx = pix.ravel()
            dd = d[idx]
            o = C - w.center
            a = dd[:, 0] ** 2 + dd[:, 2] ** 2
            b = o[0] * dd[:, 0] + o[2] * dd[:, 2]
            c = o[0] ** 2 + o[2] ** 2 - w.radius ** 2
            disc = b * b - a * c
            t = (-b + np.sqrt(np.maximum(disc, 0.0))) / a
            ok = (disc >= 0) & (a > 0) & (t > _EPS_T)
            P = C + t[:, None] * dd
            nn = np.stack([w.center[0] - P[:, 0], np.zeros(len(idx)),
                           w.center[2] - P[:, 2]], axis=-1)
            nn /= np.linalg.norm(nn, axis=-1, keepdims=True)
            ang = np.arctan2(P[:, 0] - w.center[0], P[:, 2] - w.center[2])
            s = np.floor(ang * w.radius / w.cell) + np.floor(P[:, 1] / w.cell)
            col = np.where((s.astype(np.int64) % 2 == 0)[:, None], w.color_a, w.color_b)
            take(idx[ok], t[ok], nn[ok], col[ok], oid)
            oid += 1
        for p in scene.planes:
            idx = pix.ravel()
            dd = d[idx]
            den = dd @ p.normal
            t = ((p.point - C) @ p.normal) / den
            ok = (np.abs(den) > 1e-12) & (t > _EPS_T)
            P = C + t[:, None] * dd
            if p.square > 0:
                q = P - p.point
                s = np.floor(q @ p.u_axis / p.square) + np.floor(q @ p.v_axis / p.square)
                col = np.where((s.astype(np.int64) % 2 == 0)[:, None], p.color_a, p.color_b)
            else:
                col = np.broadcast_to(p.color_a, (len(idx), 3))
            nn = np.broadcast_to(p.normal, (len(idx), 3))
            take(idx[ok], t[ok], nn[ok], col[ok], oid)
            oid += 1
        for s in scene.spheres:
            bb = _bbox_pixels(cam, s.center, s.radius)
            if bb is not None:
                u0, u1, v0, v1 = bb
                idx = pix[v0:v1, u0:u1].ravel()
                dd = d[idx]
                o = C - s.center
                a = np.einsum("ij,ij->i", dd, dd)
                b = dd @ o
                c = o @ o - s.radius ** 2
                disc = b * b - a * c
                t = (-b - np.sqrt(np.maximum(disc, 0.0))) / a
                ok = (disc >= 0) & (t > _EPS_T)
                P = C + t[:, None] * dd
                nn = (P - s.center) / s.radius
                take(idx[ok], t[ok], nn[ok], s.albedo, oid)
            oid += 1
        for bx in scene.boxes:
            bb = _bbox_pixels(cam, bx.center, float(np.linalg.norm(bx.half)))
            if bb is not None:
                u0, u1, v0, v1 = bb
                idx = pix[v0:v1, u0:u1].ravel()
                dd = d[idx]
                cs, sn = math.cos(bx.yaw), math.sin(bx.yaw)
                # world -> box frame: rotate by -yaw about y
                Rb = np.array([[cs, 0.0, -sn], [0.0, 1.0, 0.0], [sn, 0.0, cs]])
                o = Rb @ (C - bx.center)
                dl = dd @ Rb.T
                t1 = (-bx.half - o) / dl
                t2 = (bx.half - o) / dl
                tn = np.minimum(t1, t2)
                tf = np.maximum(t1, t2)
                tmin = np.max(tn, axis=1)
                tmax = np.min(tf, axis=1)
                ok = (tmax >= tmin) & (tmin > _EPS_T)
                ax = np.argmax(tn, axis=1)
                nl = np.zeros_like(dl)
                rows = np.arange(len(idx))
                nl[rows, ax] = -np.sign(dl[rows, ax])
                nn = nl @ Rb            # box frame -> world: Rb.T @ n
                take(idx[ok], tmin[ok], nn[ok], bx.albedo, oid)
            oid += 1

    hit = obj >= 0
    # face the normal towards the ray
    flip = np.einsum("ij,ij->i", nrm, d) > 0
    nrm[flip] *= -1.0
    L = scene.light_to / np.linalg.norm(scene.light_to)
    lam = np.maximum(0.0, nrm @ L)
    shade = scene.ambient + (1.0 - scene.ambient) * lam
    rgb = alb * shade[:, None]
    rgb[~hit] = 0.0
    P = C + np.where(hit, tbest, 0.0)[:, None] * d
    return {
        "rgb": rgb.reshape(H, W, 3),
        "z": tbest.reshape(H, W),
        "obj": obj.reshape(H, W),
        "normal": nrm.reshape(H, W, 3),
        "point": P.reshape(H, W, 3),
    }


def quantise(rend, max_mm: int = 65535):
    """RGB8 and uint16-mm depth from a render (0 = no depth)."""
    rgb8 = np.clip(np.floor(rend["rgb"] + 0.5), 0, 255).astype(np.uint8)
    zmm = rend["z"] * 1000.0
    ok = np.isfinite(zmm) & (zmm >= 0.5) & (zmm <= max_mm)
    d = np.where(ok, np.floor(zmm + 0.5), 0).astype(np.uint16)
    return rgb8, d


def add_depth_noise(depth: np.ndarray, z_mm: np.ndarray, rng: np.random.Generator,
                    sigma: float = 0.01, dropout: float = 0.05,
                    r_lo: float = 2.0, r_hi: float = 10.0) -> np.ndarray:
    """Multiplicative Gaussian depth noise plus zeroed discs (stereo dropouts).

    ``d = round(z * (1 + sigma * N(0, 1)))`` clamped to [1, 65535] where the
    true depth is valid; then discs of radius U(r_lo, r_hi) px at uniform
    random centres are zeroed until ``dropout`` of all pixels are 0.
    """
    H, W = depth.shape
    out = depth.copy()
    valid = depth > 0
    noisy = np.floor(z_mm * (1.0 + sigma * rng.standard_normal(depth.shape)) + 0.5)
    noisy = np.clip(np.nan_to_num(noisy, nan=0.0, posinf=0.0), 1, 65535)
    out[valid] = noisy[valid].astype(np.uint16)
    target = int(math.ceil(dropout * H * W))
    yy, xx = np.mgrid[0:H, 0:W]
    zeros = int(np.count_nonzero(out == 0))
    while zeros < target:
        cy = rng.uniform(0, H)
        cx = rng.uniform(0, W)
        r = rng.uniform(r_lo, r_hi)
        y0, y1 = max(0, int(cy - r) - 1), min(H, int(cy + r) + 2)
        x0, x1 = max(0, int(cx - r) - 1), min(W, int(cx + r) + 2)
        sub = out[y0:y1, x0:x1]
        m = (yy[y0:y1, x0:x1] - cy) ** 2 + (xx[y0:y1, x0:x1] - cx) ** 2 <= r * r
        zeros += int(np.count_nonzero(m & (sub != 0)))
        sub[m] = 0
    return out


def frames_for(scene: Scene, cams: Sequence[Camera], noise_seed: Optional[int] = None,
               sigma: float = 0.01, dropout: float = 0.05):
    """Render every camera: returns rgb (K, H, W, 3) u8 and depth (K, H, W) u16.

    All cameras must share one resolution. With ``noise_seed`` the depth noise
    model of :func:`add_depth_noise` is applied per camera.
    """
    H, W = cams[0].height, cams[0].width
    K = len(cams)
    rgb = np.zeros((K, H, W, 3), dtype=np.uint8)
    dep = np.zeros((K, H, W), dtype=np.uint16)
    rng = np.random.default_rng(noise_seed) if noise_seed is not None else None
    for k, c in enumerate(cams):
        assert (c.height, c.width) == (H, W)
        r = render(scene, c)
        rgb[k], dep[k] = quantise(r)
        if rng is not None:
            dep[k] = add_depth_noise(dep[k], r["z"] * 1000.0, rng, sigma, dropout)
    return rgb, dep


def layered_frames(bg_scene: Scene, actors: Sequence[Sphere], cams: Sequence[Camera],
                   noise_seed: Optional[int] = None, sigma: float = 0.01, dropout: float = 0.05):
    """Frames of a static background scene with moving foreground actors.

    The live frames render background + actors: RGB8 colour everywhere;
    depth (noise model of :func:`add_depth_noise` with ``noise_seed``) where
    an actor is hit, ``DEPTH_BG`` where the background is hit, 0 where
    nothing is.  The background model is the exact, noise-free depth of
    ``bg_scene`` alone (the off-line model of the static set).  The actors
    must be the scene's only spheres.  Returns rgb (K, H, W, 3) u8, live
    depth (K, H, W) u16, model depth (K, H, W) u16 and the actor mask
    (K, H, W) bool.
    """
    assert not bg_scene.spheres
    full = Scene(spheres=list(actors), boxes=bg_scene.boxes, planes=bg_scene.planes,
                 walls=bg_scene.walls, light_to=bg_scene.light_to, ambient=bg_scene.ambient)
    first = len(full.walls) + len(full.planes)           # render() numbers walls, planes, spheres, boxes
    H, W = cams[0].height, cams[0].width
    K = len(cams)
    rgb = np.zeros((K, H, W, 3), np.uint8)
    live = np.zeros((K, H, W), np.uint16)
    model = np.zeros((K, H, W), np.uint16)
    fg = np.zeros((K, H, W), bool)
    rng = np.random.default_rng(noise_seed) if noise_seed is not None else None
    for k, c in enumerate(cams):
        assert (c.height, c.width) == (H, W)
        r = render(full, c)
        rgb[k], d = quantise(r)
        if rng is not None:
            d = add_depth_noise(d, r["z"] * 1000.0, rng, sigma, dropout)
        fg[k] = (r["obj"] >= first) & (r["obj"] < first + len(actors))
        hit_bg = (r["obj"] >= 0) & ~fg[k]
        live[k] = np.where(fg[k], d, np.where(hit_bg, DEPTH_BG, 0))
        _, model[k] = quantise(render(bg_scene, c), max_mm=DEPTH_BG - 1)
    return rgb, live, model, fg


def scene_layered(seed: int, n_actors: int = 8, n_props: int = 6, half: float = 0.6,
                  floor_y: float = 0.5, wall_radius: float = 4.0):
    """A static set (checker floor, cylindrical wall, ``n_props`` yawed boxes
    with edges 0.2-0.6 m standing on the floor 2.5-3.5 m from the centre,
    within 60 deg of +z, i.e. behind the centre for cameras on the -z side)
    and ``n_actors`` spheres (r 0.1-0.3 m) inside a cube of side ``2*half``
    around the origin, so that from the rig the set is always behind the
    actors (stacking the FG layer over the BG layer is then exact).
    Returns (set, actors)."""
    rng = np.random.default_rng(seed)
    boxes = []
    for _ in range(n_props):
        e = rng.uniform(0.2, 0.6, 3)
        rr, ph = rng.uniform(2.5, 3.5), math.radians(rng.uniform(-60.0, 60.0))
        ctr = np.array([rr * math.sin(ph), floor_y - e[1] / 2, rr * math.cos(ph)])
        boxes.append(Box(ctr, e / 2, rng.uniform(0, math.pi), rng.uniform(0, 255, 3)))
    actors = []
    for _ in range(n_actors):
        r = rng.uniform(0.1, 0.3)
        ctr = np.array([rng.uniform(-half, half), rng.uniform(-half, floor_y - r),
                        rng.uniform(-half, half)])
        actors.append(Sphere(ctr, r, rng.uniform(0, 255, 3)))
    floor = Plane(np.array([0.0, floor_y, 0.0]), np.array([0.0, -1.0, 0.0]),
                  rng.uniform(60, 230, 3), rng.uniform(20, 120, 3), 0.25,
                  u_axis=np.array([1.0, 0.0, 0.0]), v_axis=np.array([0.0, 0.0, 1.0]))
    wall = CylinderWall(np.zeros(3), wall_radius, rng.uniform(90, 255, 3),
                        rng.uniform(20, 140, 3), 0.3)
    return Scene(boxes=boxes, planes=[floor], walls=[wall]), actors


# --------------------------------------------------------------------------
# rigs and trajectories
# --------------------------------------------------------------------------

def rig_parallel(n: int, width: int, height: int, f: float, baseline_m: float,
                 z0: float = 0.0) -> List[Camera]:
    """``n`` cameras on the x axis, ``baseline_m`` apart, centred on x = 0,
    all looking along +z with identity rotation."""
    xs = (np.arange(n) - (n - 1) / 2.0) * baseline_m
    cams = []
    for x in xs:
        R = np.eye(3)
        c = np.array([x, 0.0, z0])
        cams.append(Camera(width, height, f, f, (width - 1) / 2.0, (height - 1) / 2.0,
                           R, -R @ c))
    return cams


def arc_view(phi_deg: float, radius: float, width: int, height: int, f: float,
             center=(0.0, 0.0, 0.0)) -> Camera:
    """Camera on a horizontal arc around ``center``; phi = 0 is at -z looking +z."""
    ph = math.radians(phi_deg)
    O = np.asarray(center, dtype=np.float64)
    pos = O + radius * np.array([math.sin(ph), 0.0, -math.cos(ph)])
    return look_at_camera(pos, O, width, height, f)


def rig_arc(n: int, span_deg: float, radius: float, width: int, height: int,
            f: float) -> List[Camera]:
    """``n`` cameras evenly spaced over an arc of ``span_deg`` degrees."""
    if n == 1:
        return [arc_view(0.0, radius, width, height, f)]
    phis = -span_deg / 2.0 + np.arange(n) * span_deg / (n - 1)
    return [arc_view(float(p), radius, width, height, f) for p in phis]


def trajectory_arc(frames: int, amp_deg: float, radius: float, width: int,
                   height: int, f: float, period: Optional[int] = None) -> List[Camera]:
    """Smooth swing: phi(t) = amp * sin(2 pi t / period) on the rig's arc."""
    period = frames if period is None else period
    return [arc_view(amp_deg * math.sin(2.0 * math.pi * t / period), radius,
                     width, height, f) for t in range(frames)]


# --------------------------------------------------------------------------
# scenes
# --------------------------------------------------------------------------

def scene_fronto_plane(z_m: float, color_a=(200, 60, 40), color_b=(30, 90, 220),
                       square: float = 0.1) -> Scene:
    """A single fronto-parallel textured plane at depth ``z_m``."""
    pl = Plane(np.array([0.0, 0.0, z_m]), np.array([0.0, 0.0, -1.0]),
               np.array(color_a, float), np.array(color_b, float), square)
    return Scene(planes=[pl])


def scene_spheres_plane(seed: int, cam_for_frustum: Camera, n_spheres: int = 3,
                        plane_z: float = 2.0) -> Scene:
    """Three Lambertian spheres (radius U(0.2, 0.4) m, centres at z in
    [1.2, 1.7] m inside the frustum, uniform random colours) in front of a
    checker-textured plane (100 mm squares, two random colours) at 2.0 m."""
    rng = np.random.default_rng(seed)
    ca = rng.uniform(0, 255, 3)
    cb = rng.uniform(0, 255, 3)
    pl = Plane(np.array([0.0, 0.0, plane_z]), np.array([0.0, 0.0, -1.0]), ca, cb, 0.1)
    sph = []
    c = cam_for_frustum
    for _ in range(n_spheres):
        r = rng.uniform(0.2, 0.4)
        z = rng.uniform(1.2, 1.7)
        x = rng.uniform(-0.8, 0.8) * c.cx * z / c.fx
        y = rng.uniform(-0.8, 0.8) * c.cy * z / c.fy
        ctr = c.R.T @ (np.array([x, y, z]) - c.t)
        sph.append(Sphere(ctr, r, rng.uniform(0, 255, 3)))
    return Scene(spheres=sph, planes=[pl])


def scene_random_objects(seed: int, n_objects: int = 20, half: float = 0.6,
                         floor_y: float = 0.5, wall_radius: float = 4.0) -> Scene:
    """Random spheres (r 0.05-0.25 m) and yawed boxes (edges 0.1-0.4 m) in a
    cube of side ``2*half`` around the origin, a checker floor at
    y = ``floor_y`` and a cylindrical checker wall enclosing the rig."""
    rng = np.random.default_rng(seed)
    sph, boxes = [], []
    for _ in range(n_objects):
        col = rng.uniform(0, 255, 3)
        if rng.uniform() < 0.5:
            r = rng.uniform(0.05, 0.25)
            ctr = np.array([rng.uniform(-half, half),
                            rng.uniform(-half, floor_y - r),
                            rng.uniform(-half, half)])
            sph.append(Sphere(ctr, r, col))
        else:
            e = rng.uniform(0.1, 0.4, 3)
            ctr = np.array([rng.uniform(-half, half),
                            rng.uniform(-half, floor_y - e[1] / 2),
                            rng.uniform(-half, half)])
            boxes.append(Box(ctr, e / 2, rng.uniform(0, math.pi), col))
    floor = Plane(np.array([0.0, floor_y, 0.0]), np.array([0.0, -1.0, 0.0]),
                  rng.uniform(60, 230, 3), rng.uniform(20, 120, 3), 0.25,
                  u_axis=np.array([1.0, 0.0, 0.0]), v_axis=np.array([0.0, 0.0, 1.0]))
    wall = CylinderWall(np.zeros(3), wall_radius, rng.uniform(90, 255, 3),
                        rng.uniform(20, 140, 3), 0.3)
    return Scene(spheres=sph, boxes=boxes, planes=[floor], walls=[wall])


# --------------------------------------------------------------------------
# named workloads (the paper's rig shapes, synthetic content)
# --------------------------------------------------------------------------

def workload(name: str, seed: Optional[int] = None, scale: float = 1.0) -> dict:
    """Named synthetic workloads.

    * ``plain_2cam_320x240``: two parallel cameras 320x240, f = 300 px,
      baseline 100 mm; three spheres over a textured plane at 2 m; one view
      midway between the cameras; no depth noise. Seed 1.
    * ``plain_9cam_1280x720``: nine cameras 1280x720 (f = 1000 px) on a 90 deg
      arc of radius 1.5 m facing the centre; 20 random spheres and boxes, a
      floor and a wall; 1 % multiplicative depth noise and 5 % zeroed discs;
      views along phi(t) = 22.5 deg sin(2 pi t / 300). Seed 2.
    * ``plain_18cam_1920x1080``: 18 cameras 1920x1080 (f = 1500 px) on a 180 deg
      arc of radius 2 m, noise as above, the same swing trajectory. Seed 5.
    * ``layered_9cam_1280x720``: the 9-camera rig and views of
      ``plain_9cam_1280x720`` over a static set (floor, wall, 6 boxes) with 8
      sphere actors; live depth only on the actors (noise as above), the
      set signalled as background, and an exact background depth model.
      Seed 3.  Adds ``bg`` (model depth) and ``fg`` (actor mask).

    ``scale`` < 1 shrinks every resolution and focal length (for small cases).
    Returns dict(cams, rgb, depth, views, look_at, scene, name).
    """
    if name == "plain_2cam_320x240":
        seed = 1 if seed is None else seed
        W, H, f = int(round(320 * scale)), int(round(240 * scale)), 300.0 * scale
        cams = rig_parallel(2, W, H, f, 0.1)
        view = rig_parallel(1, W, H, f, 0.1)[0]
        scene = scene_spheres_plane(seed, view)
        rgb, dep = frames_for(scene, cams)
        views = [view]
        look_at = np.array([0.0, 0.0, 2.0])
    elif name == "layered_9cam_1280x720":
        seed = 3 if seed is None else seed
        W, H, f = int(round(1280 * scale)), int(round(720 * scale)), 1000.0 * scale
        cams = rig_arc(9, 90.0, 1.5, W, H, f)
        bg_scene, actors = scene_layered(seed)
        rgb, dep, bg, fg = layered_frames(bg_scene, actors, cams, noise_seed=seed + 1000)
        views = trajectory_arc(300, 22.5, 1.5, W, H, f)
        scene = Scene(spheres=list(actors), boxes=bg_scene.boxes, planes=bg_scene.planes,
                      walls=bg_scene.walls)
        return {"name": name, "cams": cams, "rgb": rgb, "depth": dep, "views": views,
                "look_at": np.zeros(3), "scene": scene, "bg_scene": bg_scene, "actors": actors,
                "bg": bg, "fg": fg}
    elif name in ("plain_9cam_1280x720", "plain_18cam_1920x1080"):
        if name == "plain_9cam_1280x720":
            seed = 2 if seed is None else seed
            K, W, H, f, span, radius = 9, 1280, 720, 1000.0, 90.0, 1.5
        else:
            seed = 5 if seed is None else seed
            K, W, H, f, span, radius = 18, 1920, 1080, 1500.0, 180.0, 2.0
        W, H, f = int(round(W * scale)), int(round(H * scale)), f * scale
        cams = rig_arc(K, span, radius, W, H, f)
        scene = scene_random_objects(seed)
        rgb, dep = frames_for(scene, cams, noise_seed=seed + 1000)
        views = trajectory_arc(300, 22.5, radius, W, H, f)
        look_at = np.zeros(3)
    else:
        raise KeyError(name)
    return {"name": name, "cams": cams, "rgb": rgb, "depth": dep, "views": views,
            "look_at": look_at, "scene": scene}
