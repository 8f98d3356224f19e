"""Seeded synthetic multi-camera RGB-D scenes.

This module only manufactures inputs: it places pinhole cameras, ray-casts analytic
primitives (planes, spheres, boxes, a room), and adds sensor noise, invalid pixels,
flying pixels, a confidence image and a colour image.  It contains none of the fusion
method's arithmetic (no gating, no consistency, no hashing, no fusion), so it can feed
both the CUDA path and the CPU oracle with identical bytes.

Camera convention (shared with the C-ABI): ``x_cam = R @ x_world + t`` with the camera
looking along +z, x to the right and y down; a pixel (x, y) has its centre at integer
coordinates.  Depth is z-depth (distance along the optical axis), not ray length.

Workload recipes (sizes follow the paper's 1-8 camera RGB-D rigs, Sec. III.2 Table III,
scaled up to the rig sizes the fusion path is benchmarked on):

* ``config1``: 2 cameras 160x120 float32 metres, ring r=2 m at 1 m height, 60 deg apart,
  plane z=0 plus a 0.4 m sphere at (0, 0, 0.4); noise N(0, (0.002 z^2)^2); 2 % of the
  pixels zeroed; seed 0.
* ``config2``: 4 cameras 640x480 uint16 mm, ring r=3 m at 1.5 m height, six boxes or
  spheres (0.2-0.8 m) on the ground, one sphere moving at 0.5 m/s (30 fps); noise
  0.0015 z^2; 1 % flying pixels at depth edges.
* ``config3``: 8 cameras 1280x720 uint16 mm, fx=fy=900, hemisphere r=4 m (elevations
  20-60 deg), ground plus 20 primitives placed from near the cameras to the centre.
* ``config4``: 2/8/16/32 cameras 1024x1024 uint16 mm, fx=fy=512 (90 deg FoV), Fibonacci
  placement on a 5 m sphere looking inward, a 16 m room (walls 8 m from the centre) plus
  spheres about 1 m in front of the rig.
* ``serving_rigs``: 2-24 cameras, 320x240 .. 1920x1080, fx = 0.714 W.

Seeds: frame ``f`` of config ``c`` draws its noise from ``1000*c + f`` (config 1 uses
seed 0); the scene layout of config ``c`` uses seed ``1000*c + 999``.
"""
from __future__ import annotations

import warnings
from dataclasses import dataclass
from typing import List, Optional, Sequence

import numpy as np

__all__ = [
    "Camera", "Rig", "Frame", "Plane", "Sphere", "Box", "Room",
    "look_at", "ring_rig", "render_frame", "config1", "config2", "config3", "config4",
    "serving_rigs", "serving_frame", "config_frame", "tiny_rig", "random_frame",
]


@dataclass
class Camera:
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    R: np.ndarray  # (3, 3) camera-from-world rotation
    t: np.ndarray  # (3,)  x_cam = R x_world + t

    @property
    def centre(self) -> np.ndarray:
        return -self.R.T @ self.t


@dataclass
class Rig:
    cameras: List[Camera]
    depth_format: str = "u16"      # "u16" (integer units) or "f32"
    depth_scale: float = 0.001     # metres per depth unit

    @property
    def n_cams(self) -> int:
        return len(self.cameras)

    @property
    def n_pixels(self) -> int:
        return int(sum(c.width * c.height for c in self.cameras))


@dataclass
class Frame:
    depth: List[np.ndarray]            # (H, W) uint16 or float32
    conf: List[np.ndarray]             # (H, W) float32
    rgb: List[np.ndarray]              # (H, W, 3) uint8
    z_true: Optional[List[np.ndarray]] = None   # (H, W) float64 noiseless z, 0 = no hit
    surface_id: Optional[List[np.ndarray]] = None  # (H, W) int16 primitive index, -1 = none

    def input_bytes(self) -> int:
        return int(sum(d.nbytes + c.nbytes + r.nbytes
                       for d, c, r in zip(self.depth, self.conf, self.rgb)))


# ----------------------------------------------------------------------------- primitives
@dataclass
class Plane:
    normal: Sequence[float]
    offset: float  # plane: normal . x = offset


@dataclass
class Sphere:
    centre: Sequence[float]
    radius: float


@dataclass
class Box:
    lo: Sequence[float]
    hi: Sequence[float]


@dataclass
class Room:
    """Axis-aligned box seen from the inside (the cameras sit within it)."""
    lo: Sequence[float]
    hi: Sequence[float]


def look_at(centre, target, fx, fy, cx, cy, width, height, up=(0.0, 0.0, 1.0)) -> Camera:
    """Pinhole camera at ``centre`` whose optical axis passes through ``target``."""
    c = np.asarray(centre, dtype=np.float64)
    fwd = np.asarray(target, dtype=np.float64) - c
    fwd /= np.linalg.norm(fwd)
    upv = np.asarray(up, dtype=np.float64)
    right = np.cross(fwd, upv)
    if np.linalg.norm(right) < 1e-6:          # looking straight up or down
        right = np.cross(fwd, np.array([0.0, 1.0, 0.0]))
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    R = np.stack([right, down, fwd])
    t = -R @ c
    return Camera(float(fx), float(fy), float(cx), float(cy), int(width), int(height), R, t)


def ring_rig(n, radius, height, fx, fy, cx, cy, width, height_px, start_deg=0.0, step_deg=None,
             depth_format="u16", depth_scale=0.001) -> Rig:
    step = 360.0 / n if step_deg is None else step_deg
    cams = []
    for k in range(n):
        a = np.deg2rad(start_deg + k * step)
        cams.append(look_at((radius * np.cos(a), radius * np.sin(a), height), (0, 0, 0),
                            fx, fy, cx, cy, width, height_px))
    return Rig(cams, depth_format, depth_scale)


# ----------------------------------------------------------------------------- ray casting
def _pixel_rays(cam: Camera):
    """Unnormalised world-space ray per pixel centre, scaled so that its camera-z is 1.

    Walking ``t`` along such a ray from the camera centre reaches a point whose z-depth
    is exactly ``t``.
    """
    xs = (np.arange(cam.width, dtype=np.float64) - cam.cx) / cam.fx
    ys = (np.arange(cam.height, dtype=np.float64) - cam.cy) / cam.fy
    d_cam = np.empty((cam.height, cam.width, 3))
    d_cam[..., 0] = xs[None, :]
    d_cam[..., 1] = ys[:, None]
    d_cam[..., 2] = 1.0
    return d_cam @ cam.R  # rows times R == (R^T d)^T


def _hit_plane(o, d, p: Plane):
    n = np.asarray(p.normal, dtype=np.float64)
    n = n / np.linalg.norm(n)
    denom = d @ n
    with np.errstate(divide="ignore", invalid="ignore"):
        t = (p.offset - o @ n) / denom
    t = np.where((np.abs(denom) > 1e-12) & (t > 1e-9), t, np.inf)
    normal = np.broadcast_to(n, d.shape)
    return t, normal


def _hit_sphere(o, d, s: Sphere):
    c = np.asarray(s.centre, dtype=np.float64)
    oc = o - c
    a = np.einsum("...k,...k->...", d, d)
    b = d @ oc
    cc = oc @ oc - s.radius ** 2
    disc = b * b - a * cc
    with np.errstate(invalid="ignore"):
        sq = np.sqrt(np.maximum(disc, 0.0))
    t = (-b - sq) / a
    t = np.where((disc >= 0) & (t > 1e-9), t, np.inf)
    p = o + np.where(np.isfinite(t), t, 0.0)[..., None] * d
    normal = (p - c) / s.radius
    return t, normal


def _slabs(o, d, lo, hi):
    with np.errstate(divide="ignore", invalid="ignore"):
        t1 = (lo - o) / d
        t2 = (hi - o) / d
    tn = np.minimum(t1, t2)
    tf = np.maximum(t1, t2)
    tn = np.where(np.isnan(tn), -np.inf, tn)
    tf = np.where(np.isnan(tf), np.inf, tf)
    return tn, tf


def _hit_box(o, d, b: Box):
    lo = np.asarray(b.lo, dtype=np.float64)
    hi = np.asarray(b.hi, dtype=np.float64)
    tn, tf = _slabs(o, d, lo, hi)
    t_enter = tn.max(axis=-1)
    t_exit = tf.min(axis=-1)
    axis = tn.argmax(axis=-1)
    t = np.where((t_exit >= t_enter) & (t_enter > 1e-9), t_enter, np.inf)
    normal = np.zeros(d.shape)
    sign = -np.sign(np.take_along_axis(d, axis[..., None], axis=-1))[..., 0]
    np.put_along_axis(normal, axis[..., None], sign[..., None], axis=-1)
    return t, normal


def _hit_room(o, d, r: Room):
    lo = np.asarray(r.lo, dtype=np.float64)
    hi = np.asarray(r.hi, dtype=np.float64)
    tn, tf = _slabs(o, d, lo, hi)
    t_exit = tf.min(axis=-1)
    axis = tf.argmin(axis=-1)
    t = np.where(t_exit > 1e-9, t_exit, np.inf)
    normal = np.zeros(d.shape)
    sign = -np.sign(np.take_along_axis(d, axis[..., None], axis=-1))[..., 0]
    np.put_along_axis(normal, axis[..., None], sign[..., None], axis=-1)
    return t, normal


_HIT = {Plane: _hit_plane, Sphere: _hit_sphere, Box: _hit_box, Room: _hit_room}


def _bounding_sphere(p):
    if isinstance(p, Sphere):
        return np.asarray(p.centre, dtype=np.float64), float(p.radius)
    if isinstance(p, Box):
        lo = np.asarray(p.lo, dtype=np.float64)
        hi = np.asarray(p.hi, dtype=np.float64)
        return (lo + hi) / 2, float(np.linalg.norm(hi - lo) / 2)
    return None, None


def _pixel_window(cam: Camera, p):
    """Conservative pixel rectangle (y0, y1, x0, x1) that can see primitive ``p``."""
    full = (0, cam.height, 0, cam.width)
    c, rho = _bounding_sphere(p)
    if c is None:
        return full
    q = cam.R @ c + cam.t
    corners = q[None, :] + rho * np.array([[sx, sy, sz] for sx in (-1, 1) for sy in (-1, 1)
                                          for sz in (-1, 1)], dtype=np.float64)
    if np.any(corners[:, 2] <= 1e-6):
        return full
    u = cam.fx * corners[:, 0] / corners[:, 2] + cam.cx
    v = cam.fy * corners[:, 1] / corners[:, 2] + cam.cy
    x0 = int(np.clip(np.floor(u.min()) - 1, 0, cam.width))
    x1 = int(np.clip(np.ceil(u.max()) + 2, 0, cam.width))
    y0 = int(np.clip(np.floor(v.min()) - 1, 0, cam.height))
    y1 = int(np.clip(np.ceil(v.max()) + 2, 0, cam.height))
    return y0, y1, x0, x1


def ray_cast(cam: Camera, prims) -> tuple:
    """Nearest hit per pixel: (z-depth, unit normal, world hit point, primitive id, rays)."""
    d = _pixel_rays(cam)
    o = cam.centre
    z = np.full(d.shape[:2], np.inf)
    normal = np.zeros(d.shape)
    sid = np.full(d.shape[:2], -1, dtype=np.int16)
    for k, p in enumerate(prims):
        y0, y1, x0, x1 = _pixel_window(cam, p)
        if y1 <= y0 or x1 <= x0:
            continue
        win = (slice(y0, y1), slice(x0, x1))
        t, n = _HIT[type(p)](o, d[win], p)
        closer = t < z[win]
        z[win] = np.where(closer, t, z[win])
        normal[win] = np.where(closer[..., None], n, normal[win])
        sid[win] = np.where(closer, np.int16(k), sid[win])
    hit = np.isfinite(z)
    pts = o + np.where(hit, z, 0.0)[..., None] * d
    return np.where(hit, z, 0.0), normal, pts, sid, d


# ----------------------------------------------------------------------------- sensor model
def _colour_hash(pts: np.ndarray) -> np.ndarray:
    """uint8 RGB from the 1 cm lattice cell of the true surface point (splitmix64 mixing)."""
    q = np.rint(pts / 0.01).astype(np.int64).astype(np.uint64)
    h = (q[..., 0] * np.uint64(0x9E3779B97F4A7C15)) ^ (q[..., 1] * np.uint64(0xC2B2AE3D27D4EB4F)) \
        ^ (q[..., 2] * np.uint64(0x165667B19E3779F9))
    h ^= h >> np.uint64(30)
    h *= np.uint64(0xBF58476D1CE4E5B9)
    h ^= h >> np.uint64(27)
    h *= np.uint64(0x94D049BB133111EB)
    h ^= h >> np.uint64(31)
    rgb = np.stack([(h >> np.uint64(s)) & np.uint64(0xFF) for s in (0, 8, 16)], axis=-1)
    return rgb.astype(np.uint8)


def _depth_edges(z_true):
    """Depth-edge pixels (4-neighbourhood range above 0.1 m) with their fg/bg depths."""
    zt = np.where(z_true > 0, z_true, np.nan)
    pad = np.pad(zt, 1, constant_values=np.nan)
    nb = np.stack([pad[1:-1, :-2], pad[1:-1, 2:], pad[:-2, 1:-1], pad[2:, 1:-1], zt])
    with np.errstate(invalid="ignore"), warnings.catch_warnings():
        warnings.simplefilter("ignore", RuntimeWarning)
        zmin = np.nanmin(nb, axis=0)
        zmax = np.nanmax(nb, axis=0)
    edge = np.isfinite(zmin) & (zmax - zmin > 0.1)
    idx = np.flatnonzero(edge)
    return idx, zmin.ravel()[idx], zmax.ravel()[idx]


def _flying_pixels(edges, z_noisy, frac, rng):
    """Replace ``frac`` of the pixels, drawn among depth-edge pixels, by a fg/bg blend."""
    idx, zmin, zmax = edges
    H, W = z_noisy.shape
    n_fly = min(idx.size, int(round(frac * H * W)))
    if n_fly == 0:
        return z_noisy
    pick = rng.choice(idx.size, size=n_fly, replace=False)
    mix = rng.uniform(0.0, 1.0, size=n_fly)
    out = z_noisy.copy().ravel()
    out[idx[pick]] = zmin[pick] + mix * (zmax[pick] - zmin[pick])
    return out.reshape(H, W)


def render_frame(rig: Rig, prims, seed: int, noise_k: float = 0.0015, zero_frac: float = 0.0,
                 flying_frac: float = 0.0, conf_jitter: float = 0.05, keep_truth: bool = False,
                 noiseless: bool = False, cache: Optional[dict] = None) -> Frame:
    """Render depth/confidence/colour for every camera of ``rig``.

    * depth: z-depth + N(0, (noise_k z^2)^2), encoded as uint16 (rounded depth units,
      0 = invalid) or float32 (0 = invalid).
    * confidence: clamp(1 - 0.5 * cos(grazing angle) + U(-conf_jitter, conf_jitter), 0, 1),
      with cos(grazing) = sqrt(1 - (n . r)^2) for surface normal n and unit view ray r:
      frontal views give about 1, grazing views about 0.5.
    * colour: hash of the 1 cm lattice cell of the true surface point.

    ``cache`` (a dict) keeps the ray-cast of each camera between frames of a static scene.
    """
    rng = np.random.default_rng(seed)
    depth, conf, rgb, ztrue, sids = [], [], [], [], []
    for ci, cam in enumerate(rig.cameras):
        if cache is not None and ci in cache:
            z, n, pts, sid, d, cos_graze, col, edges = cache[ci]
        else:
            z, n, pts, sid, d = ray_cast(cam, prims)
            rhat = d / np.linalg.norm(d, axis=-1, keepdims=True)
            ndotr = np.einsum("...k,...k->...", n, rhat)
            cos_graze = np.sqrt(np.clip(1.0 - ndotr * ndotr, 0.0, 1.0))
            col = np.where((z > 0)[..., None], _colour_hash(pts), 0).astype(np.uint8)
            edges = _depth_edges(z) if flying_frac > 0 else None
            if cache is not None:
                cache[ci] = (z, n, pts, sid, d, cos_graze, col, edges)
        hit = z > 0
        if noiseless:
            zn = z.copy()
        else:
            zn = z + rng.normal(0.0, 1.0, size=z.shape) * noise_k * z * z
        if flying_frac > 0:
            zn = _flying_pixels(edges if edges is not None else _depth_edges(z), zn, flying_frac, rng)
        zn = np.where(hit & (zn > 0), zn, 0.0)
        if zero_frac > 0:
            kill = rng.random(z.shape) < zero_frac
            zn = np.where(kill, 0.0, zn)
        c = 1.0 - 0.5 * cos_graze + rng.uniform(-conf_jitter, conf_jitter, size=z.shape)
        c = np.where(hit, np.clip(c, 0.0, 1.0), 0.0).astype(np.float32)
        if rig.depth_format == "u16":
            units = np.rint(zn / rig.depth_scale)
            dep = np.clip(units, 0, 65535).astype(np.uint16)
        elif rig.depth_format == "f32":
            dep = (zn / rig.depth_scale).astype(np.float32)
        else:
            raise ValueError(rig.depth_format)
        depth.append(np.ascontiguousarray(dep))
        conf.append(np.ascontiguousarray(c))
        rgb.append(np.ascontiguousarray(col))
        if keep_truth:
            ztrue.append(z)
            sids.append(sid)
    return Frame(depth, conf, rgb, ztrue if keep_truth else None, sids if keep_truth else None)


# ----------------------------------------------------------------------------- configs
def config1(keep_truth=False, noiseless=False):
    rig = ring_rig(2, 2.0, 1.0, 150.0, 150.0, 80.0, 60.0, 160, 120, start_deg=0.0, step_deg=60.0,
                   depth_format="f32", depth_scale=1.0)
    prims = [Plane((0, 0, 1), 0.0), Sphere((0.0, 0.0, 0.4), 0.4)]
    fr = render_frame(rig, prims, seed=0, noise_k=0.002, zero_frac=0.02, keep_truth=keep_truth,
                      noiseless=noiseless)
    return rig, prims, fr


def _ground_objects(rng, n, r_lo, r_hi, size_lo, size_hi):
    prims = []
    for k in range(n):
        rad = rng.uniform(r_lo, r_hi)
        ang = rng.uniform(0, 2 * np.pi)
        size = rng.uniform(size_lo, size_hi)
        x, y = rad * np.cos(ang), rad * np.sin(ang)
        if k % 2 == 0:
            prims.append(Sphere((x, y, size / 2), size / 2))
        else:
            h = size / 2
            prims.append(Box((x - h, y - h, 0.0), (x + h, y + h, size)))
    return prims


def config2(frame=0, keep_truth=False):
    rig = ring_rig(4, 3.0, 1.5, 525.0, 525.0, 320.0, 240.0, 640, 480, start_deg=45.0)
    rng = np.random.default_rng(1000 * 2 + 999)
    objs = _ground_objects(rng, 6, 0.0, 1.5, 0.2, 0.8)
    s0 = objs[0]
    moved = Sphere((s0.centre[0] + 0.5 * frame / 30.0, s0.centre[1], s0.centre[2]), s0.radius)
    prims = [Plane((0, 0, 1), 0.0), moved] + objs[1:]
    fr = render_frame(rig, prims, seed=1000 * 2 + frame, noise_k=0.0015, flying_frac=0.01,
                      keep_truth=keep_truth)
    return rig, prims, fr


def config3_rig() -> Rig:
    cams = []
    for k in range(8):
        elev = np.deg2rad(20.0 + 40.0 * k / 7.0)
        az = np.deg2rad(45.0 * k)
        c = 4.0 * np.array([np.cos(elev) * np.cos(az), np.cos(elev) * np.sin(az), np.sin(elev)])
        cams.append(look_at(c, (0, 0, 0), 900.0, 900.0, 640.0, 360.0, 1280, 720))
    return Rig(cams, "u16", 0.001)


def config3(frame=0, keep_truth=False, cache=None):
    """8 x 1280x720 hemisphere rig; the scene is static, so ``cache`` may carry the
    ray-cast between frames (only the sensor noise changes)."""
    rig = config3_rig()
    rng = np.random.default_rng(1000 * 3 + 999)
    objs = _ground_objects(rng, 20, 0.3, 3.2, 0.1, 0.6)
    prims = [Plane((0, 0, 1), 0.0)] + objs
    fr = render_frame(rig, prims, seed=1000 * 3 + frame, noise_k=0.0015, flying_frac=0.01,
                      keep_truth=keep_truth, cache=cache)
    return rig, prims, fr


def fibonacci_rig(n, radius=5.0, f=512.0, size=1024) -> Rig:
    cams = []
    golden = np.pi * (3.0 - np.sqrt(5.0))
    for i in range(n):
        z = 1.0 - 2.0 * (i + 0.5) / n
        r = np.sqrt(max(0.0, 1.0 - z * z))
        a = golden * i
        c = radius * np.array([r * np.cos(a), r * np.sin(a), z])
        cams.append(look_at(c, (0, 0, 0), f, f, size / 2, size / 2, size, size))
    return Rig(cams, "u16", 0.001)


def config4(n_cams=8, frame=0, keep_truth=False, size=1024, cache=None):
    rig = fibonacci_rig(n_cams, 5.0, 512.0 * size / 1024, size)
    rng = np.random.default_rng(1000 * 4 + 999)
    prims = [Room((-8, -8, -8), (8, 8, 8)), Box((-0.6, -0.6, -0.6), (0.6, 0.6, 0.6))]
    for _ in range(8):
        v = rng.normal(size=3)
        v /= np.linalg.norm(v)
        prims.append(Sphere(tuple(4.0 * v), rng.uniform(0.2, 0.5)))
    fr = render_frame(rig, prims, seed=1000 * 4 + frame, noise_k=0.0015, flying_frac=0.01,
                      keep_truth=keep_truth, cache=cache)
    return rig, prims, fr


_RES = [(320, 240), (640, 480), (1280, 720), (1920, 1080)]


def serving_rigs(n_rigs=12, seed=5999):
    """Rigs of 2-24 cameras on rings around a shared scene, resolution per rig, fx = 0.714 W."""
    rng = np.random.default_rng(seed)
    rigs = []
    for r in range(n_rigs):
        n = int(rng.integers(2, 25))
        w, h = _RES[int(rng.integers(0, len(_RES)))]
        f = 0.714 * w
        radius = rng.uniform(3.0, 4.5)
        rig = ring_rig(n, radius, rng.uniform(1.0, 2.5), f, f, w / 2, h / 2, w, h,
                       start_deg=rng.uniform(0, 360))
        rigs.append(rig)
    rng2 = np.random.default_rng(seed + 1)
    prims = [Plane((0, 0, 1), 0.0)] + _ground_objects(rng2, 10, 0.0, 2.0, 0.2, 0.8)
    return rigs, prims


def config_frame(spec) -> tuple:
    """(rig, frame) of a configuration named by a picklable spec: ("cfg1",), ("cfg2", f),
    ("cfg3", f) or ("cfg4", n_cams); module-level so that a process pool can render them."""
    name = spec[0]
    if name == "cfg1":
        rig, _, fr = config1()
    elif name == "cfg2":
        rig, _, fr = config2(frame=spec[1])
    elif name == "cfg3":
        rig, _, fr = config3(frame=spec[1])
    elif name == "cfg4":
        rig, _, fr = config4(n_cams=spec[1])
    else:
        raise ValueError(name)
    return rig, fr


def serving_frame(index: int, n_rigs: int = 12, seed: int = 5999) -> Frame:
    """Frame 0 of serving rig `index` (noise seed 1000*5 + index); a module-level function so
    that a process pool can render the rigs in parallel."""
    rigs, prims = serving_rigs(n_rigs, seed)
    return render_frame(rigs[index], prims, seed=1000 * 5 + index, noise_k=0.0015,
                        flying_frac=0.01)


# ----------------------------------------------------------------------------- tiny cases
def tiny_rig(n=2, width=8, height=6, depth_format="u16", depth_scale=0.001, spread_deg=30.0,
             radius=2.0, height_m=1.0, fx=None, fy=None, cx=None, cy=None) -> Rig:
    fx = width * 0.9 if fx is None else fx
    fy = width * 0.85 if fy is None else fy
    cx = (width - 1) / 2 + 0.3 if cx is None else cx
    cy = (height - 1) / 2 - 0.2 if cy is None else cy
    return ring_rig(n, radius, height_m, fx, fy, cx, cy, width, height, start_deg=10.0,
                    step_deg=spread_deg, depth_format=depth_format, depth_scale=depth_scale)


def random_frame(rig: Rig, seed: int, prims=None, noise_k=0.0015, zero_frac=0.02,
                 flying_frac=0.0):
    """A ground plane with a sphere and a box, rendered with the standard sensor model."""
    if prims is None:
        prims = [Plane((0, 0, 1), 0.0), Sphere((0.1, -0.1, 0.35), 0.35),
                 Box((-0.6, 0.2, 0.0), (-0.2, 0.6, 0.3))]
    return render_frame(rig, prims, seed=seed, noise_k=noise_k, zero_frac=zero_frac,
                        flying_frac=flying_frac)
