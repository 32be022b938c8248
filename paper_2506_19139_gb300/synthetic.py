"""Seeded synthetic scenes, cameras and query points shaped like the paper's workloads.

The paper measures on trained Tanks & Temples / Mip-NeRF 360 / DTU captures (Sec. 4); none of
them is available here, so these generators stand in for them with the shapes, sizes and value
distributions of unbounded captures: ~0.4-2.7M Gaussians (App. B, Table "Point Cloud Analysis"),
1080p-class images, a dense foreground plus a log-distributed background.

This module holds none of the compositing arithmetic. It only draws parameters from fixed
distributions and builds camera poses (look-at frames, pinhole intrinsics). Both the FP64 oracle
tests and the CUDA path consume the arrays it returns, so it is the one module they share.

Conventions of the returned arrays (float32, C-contiguous):
  means [N,3]; log_scales [N,3]; quats [N,4] as (w,x,y,z), not necessarily unit length;
  opacity_logits [N]; sh [N,(deg+1)^2,3].
  Camera: world_to_cam [3,4] row-major, OpenCV axes (x right, y down, z forward);
  fx, fy, cx, cy in pixels; width, height.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Scene:
    means: np.ndarray
    log_scales: np.ndarray
    quats: np.ndarray
    opacity_logits: np.ndarray
    sh: np.ndarray
    sh_degree: int

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def subset(self, idx) -> "Scene":
        return Scene(self.means[idx].copy(), self.log_scales[idx].copy(), self.quats[idx].copy(),
                     self.opacity_logits[idx].copy(), self.sh[idx].copy(), self.sh_degree)


@dataclasses.dataclass
class Camera:
    world_to_cam: np.ndarray  # [3,4] float32
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int

    @property
    def intr(self) -> np.ndarray:
        return np.array([self.fx, self.fy, self.cx, self.cy], dtype=np.float32)


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def _logit(p: np.ndarray) -> np.ndarray:
    return np.log(p / (1.0 - p))


def _unit_quats(rng: np.random.Generator, n: int) -> np.ndarray:
    q = rng.standard_normal((n, 4))
    return q / np.linalg.norm(q, axis=1, keepdims=True)


def _dc_from_rgb(rgb: np.ndarray) -> np.ndarray:
    # Degree-0 real SH basis value 1/(2 sqrt(pi)); DC coefficient chosen so that the
    # view-independent colour (DC term + 0.5 offset) equals the drawn rgb.
    return (rgb - 0.5) / (0.5 / math.sqrt(math.pi))


def _sh_coeffs(rng: np.random.Generator, n: int, degree: int) -> np.ndarray:
    k = (degree + 1) ** 2
    sh = np.zeros((n, k, 3))
    sh[:, 0, :] = _dc_from_rgb(rng.uniform(0.0, 1.0, (n, 3)))
    if k > 1:
        sh[:, 1:, :] = rng.normal(0.0, 0.1, (n, k - 1, 3))
    return sh


# ----------------------------------------------------------------------------- scenes

def uniform_box_scene(n: int, seed: int, half_extent: float = 1.0, log_scale_range=(0.01, 0.1),
                      opacity_range=(0.1, 0.99), sh_degree: int = 0) -> Scene:
    """Means uniform in [-h,h]^3, log-scales uniform in [ln a, ln b] per axis, uniformly random
    rotations, opacities uniform, SH as above (the tiny and differentiable configurations)."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(-half_extent, half_extent, (n, 3))
    lo, hi = log_scale_range
    log_scales = rng.uniform(math.log(lo), math.log(hi), (n, 3))
    quats = _unit_quats(rng, n)
    opac = rng.uniform(opacity_range[0], opacity_range[1], n)
    sh = _sh_coeffs(rng, n, sh_degree)
    return Scene(_f32(means), _f32(log_scales), _f32(quats), _f32(_logit(opac)), _f32(sh), sh_degree)


def unbounded_scene(n: int, seed: int, sh_degree: int = 3, fg_fraction: float = 0.7) -> Scene:
    """Unbounded-capture stand-in: a dense foreground (means N(0,I) rejection-sampled inside the
    unit sphere) plus a background at radius log-uniform in [2,100] with uniform direction. Scales
    log-normal(ln 0.02, 0.7) per axis, multiplied by the radius for background Gaussians.
    Opacities Beta(2,2)."""
    rng = np.random.default_rng(seed)
    n_fg = int(round(n * fg_fraction))
    n_bg = n - n_fg
    fg = np.empty((0, 3))
    while fg.shape[0] < n_fg:
        cand = rng.standard_normal((2 * (n_fg - fg.shape[0]) + 16, 3))
        cand = cand[np.linalg.norm(cand, axis=1) < 1.0]
        fg = np.concatenate([fg, cand], axis=0)
    fg = fg[:n_fg]
    u = rng.standard_normal((n_bg, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    r = np.exp(rng.uniform(math.log(2.0), math.log(100.0), n_bg))
    bg = u * r[:, None]
    means = np.concatenate([fg, bg], axis=0)
    scales = np.exp(rng.normal(math.log(0.02), 0.7, (n, 3)))
    scales[n_fg:] *= np.linalg.norm(bg, axis=1)[:, None]
    perm = rng.permutation(n)
    means = means[perm]
    scales = scales[perm]
    quats = _unit_quats(rng, n)
    opac = np.clip(rng.beta(2.0, 2.0, n), 1e-4, 1.0 - 1e-4)
    sh = _sh_coeffs(rng, n, sh_degree)
    return Scene(_f32(means), _f32(np.log(scales)), _f32(quats), _f32(_logit(opac)), _f32(sh), sh_degree)


def principal_frames(scene: Scene) -> np.ndarray:
    """Rotation matrices [N,3,3] whose columns are the principal axes of each Gaussian, built from
    the (w,x,y,z) quaternion. Used only to place query points; neither side reads it."""
    q = scene.quats.astype(np.float64)
    q = q / np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    R = np.empty((q.shape[0], 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - w * z)
    R[:, 0, 2] = 2 * (x * z + w * y)
    R[:, 1, 0] = 2 * (x * y + w * z)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - w * x)
    R[:, 2, 0] = 2 * (x * z - w * y)
    R[:, 2, 1] = 2 * (y * z + w * x)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def box_corner_points(scene: Scene, k_sigma: float = 3.0) -> np.ndarray:
    """Query points of the meshing workload: each Gaussian's mean plus the 8 corners of its
    +-k_sigma box in the principal frame (9 points per Gaussian), shape [9N,3], float32."""
    R = principal_frames(scene)
    s = np.exp(scene.log_scales.astype(np.float64))
    mu = scene.means.astype(np.float64)
    signs = np.array([[sx, sy, sz] for sx in (-1, 1) for sy in (-1, 1) for sz in (-1, 1)], dtype=np.float64)
    local = k_sigma * signs[None, :, :] * s[:, None, :]            # [N,8,3]
    corners = mu[:, None, :] + np.einsum("nij,nkj->nki", R, local)  # [N,8,3]
    pts = np.concatenate([mu[:, None, :], corners], axis=1).reshape(-1, 3)
    return _f32(pts)


# ----------------------------------------------------------------------------- cameras

def pinhole(width: int, height: int, fov_x_deg: float = 60.0):
    fx = 0.5 * width / math.tan(math.radians(fov_x_deg) * 0.5)
    return fx, fx, 0.5 * width, 0.5 * height


def _frame_from_forward(forward, up_hint, roll: float = 0.0) -> np.ndarray:
    f = np.asarray(forward, dtype=np.float64)
    f = f / np.linalg.norm(f)
    up = np.asarray(up_hint, dtype=np.float64)
    if abs(float(np.dot(up, f))) > 0.999:
        up = np.array([1.0, 0.0, 0.0]) if abs(f[0]) < 0.9 else np.array([0.0, 0.0, 1.0])
    right = np.cross(f, up)
    right /= np.linalg.norm(right)
    down = np.cross(f, right)
    if roll != 0.0:
        cr, sr = math.cos(roll), math.sin(roll)
        right, down = cr * right + sr * down, -sr * right + cr * down
    return np.stack([right, down, f], axis=0)  # rows: camera axes in world coordinates


def camera_from_frame(Rwc: np.ndarray, eye, width: int, height: int, fov_x_deg: float = 60.0) -> Camera:
    eye = np.asarray(eye, dtype=np.float64)
    t = -Rwc @ eye
    w2c = np.concatenate([Rwc, t[:, None]], axis=1)
    fx, fy, cx, cy = pinhole(width, height, fov_x_deg)
    return Camera(_f32(w2c), fx, fy, cx, cy, int(width), int(height))


def look_at(eye, target, width: int, height: int, fov_x_deg: float = 60.0, up=(0.0, 1.0, 0.0),
            roll: float = 0.0) -> Camera:
    # OpenCV axes: world +y up in the image means camera +y (down) points along world -y.
    fwd = np.asarray(target, dtype=np.float64) - np.asarray(eye, dtype=np.float64)
    return camera_from_frame(_frame_from_forward(fwd, up, roll), eye, width, height, fov_x_deg)


def fibonacci_sphere(n: int) -> np.ndarray:
    i = np.arange(n, dtype=np.float64) + 0.5
    phi = np.arccos(1.0 - 2.0 * i / n)
    theta = math.pi * (1.0 + math.sqrt(5.0)) * i
    return np.stack([np.cos(theta) * np.sin(phi), np.sin(theta) * np.sin(phi), np.cos(phi)], axis=1)


def _random_rotation(rng: np.random.Generator) -> np.ndarray:
    q = _unit_quats(rng, 1)[0]
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


# ----------------------------------------------------------------------------- workloads

def tiny_forward(seed: int = 0, n: int = 1000):
    """1,000 Gaussians in [-1,1]^3, log-scales U[ln .01, ln .1], opacities U(0.1,0.99), SH degree 0;
    one 64x64 camera at distance 4 looking at the origin, fov 60 deg."""
    scene = uniform_box_scene(n, seed, 1.0, (0.01, 0.1), (0.1, 0.99), 0)
    cam = look_at((0.0, 0.0, 4.0), (0.0, 0.0, 0.0), 64, 64, 60.0)
    return scene, [cam]


def differentiable_step(seed: int = 1, n: int = 100_000, res: int = 256):
    """100,000 Gaussians in [-2,2]^3 with SH degree 3; four cameras at 256x256 on a ring of radius 6."""
    scene = uniform_box_scene(n, seed, 2.0, (0.01, 0.1), (0.1, 0.99), 3)
    cams = []
    for k in range(4):
        a = k * 0.5 * math.pi
        cams.append(look_at((6.0 * math.sin(a), 0.0, 6.0 * math.cos(a)), (0, 0, 0), res, res, 60.0))
    return scene, cams


def gradient_check(seed: int = 11, n: int = 200, res: int = 32, half_extent: float = 1.0,
                   log_scale_range=(0.05, 0.3), sh_degree: int = 3, distance: float = 4.0):
    """Small scene for finite-difference gradient checks: n Gaussians seen at res x res."""
    scene = uniform_box_scene(n, seed, half_extent, log_scale_range, (0.1, 0.99), sh_degree)
    cam = look_at((0.3, 0.2, distance), (0.0, 0.0, 0.0), res, res, 60.0)
    return scene, [cam]


def unbounded_training(seed: int = 2, n: int = 1_000_000, width: int = 1920, height: int = 1080):
    """1M-Gaussian unbounded scene, one 1920x1080 camera inside the unit sphere looking outward."""
    scene = unbounded_scene(n, seed, 3)
    rng = np.random.default_rng(seed + 1000)
    while True:
        c = rng.uniform(-0.5, 0.5, 3)
        r = float(np.linalg.norm(c))
        if 0.05 < r < 0.5:
            break
    roll = rng.uniform(0.0, 2.0 * math.pi)
    Rwc = _frame_from_forward(c / r, (0.0, 1.0, 0.0), roll)
    return scene, [camera_from_frame(Rwc, c, width, height, 60.0)]


def meshing_query(seed: int = 3, n: int = 3_000_000, n_views: int = 100, width: int = 1000,
                  height: int = 750, fg_fraction: float = 0.7):
    """3M-Gaussian unbounded scene, 9 query points per Gaussian, n_views cameras at radius 3 on a
    Fibonacci sphere with jittered look-at targets. fg_fraction = 1 leaves out the background
    shell (radius 2 to 100) that surrounds the cameras."""
    scene = unbounded_scene(n, seed, 3, fg_fraction)
    pts = box_corner_points(scene, 3.0)
    rng = np.random.default_rng(seed + 1000)
    cams = []
    for p in fibonacci_sphere(n_views):
        target = rng.normal(0.0, 0.1, 3)
        cams.append(look_at(3.0 * p, target, width, height, 60.0))
    return scene, cams, pts


BATCH_RESOLUTIONS = ((512, 384), (960, 540), (1280, 720), (1600, 1064), (1920, 1080))


def batched_views(seed: int = 4, n: int = 3_000_000, n_views: int = 32):
    """3M-Gaussian unbounded scene; n_views cameras with resolutions drawn from BATCH_RESOLUTIONS,
    positions uniform in the unit ball and uniformly random orientations."""
    scene = unbounded_scene(n, seed, 3)
    rng = np.random.default_rng(seed + 1000)
    cams = []
    for _ in range(n_views):
        while True:
            c = rng.uniform(-1.0, 1.0, 3)
            if np.linalg.norm(c) < 1.0:
                break
        w, h = BATCH_RESOLUTIONS[int(rng.integers(len(BATCH_RESOLUTIONS)))]
        cams.append(camera_from_frame(_random_rotation(rng), c, w, h, 60.0))
    return scene, cams


def random_target(cams, seed: int = 7):
    rng = np.random.default_rng(seed)
    return [_f32(rng.uniform(0.0, 1.0, (3, c.height, c.width))) for c in cams]


def toward_camera_points(points: np.ndarray, cams, idx: np.ndarray, dist: float = 0.3, near: float = 0.2,
                         seed: int = 11, tries: int = 32):
    """For each points[idx[i]], a point on the segment from it to the centre of a random camera whose
    image holds the point (projection in [0,W) x [0,H) and camera depth beyond `near`), at distance
    `dist` from that centre: the far ends of edges for a level-set bisection that start at points
    inside the surface (little lies between a camera and a point next to it). Points no camera was
    found for (after `tries` draws) keep their own position. Returns (float32 [len(idx), 3], the
    camera index per point or -1)."""
    rng = np.random.default_rng(seed)
    x = points[idx].astype(np.float64)
    R = np.stack([c.world_to_cam[:, :3].astype(np.float64) for c in cams])
    t = np.stack([c.world_to_cam[:, 3].astype(np.float64) for c in cams])
    centre = -np.einsum("vji,vj->vi", R, t)
    intr = np.stack([c.intr.astype(np.float64) for c in cams])
    wh = np.array([[c.width, c.height] for c in cams], dtype=np.float64)
    view = np.full(len(idx), -1, dtype=np.int64)
    todo = np.arange(len(idx))
    for _ in range(tries):
        if todo.size == 0:
            break
        v = rng.integers(0, len(cams), todo.size)
        pc = np.einsum("nij,nj->ni", R[v], x[todo]) + t[v]
        z = pc[:, 2]
        with np.errstate(divide="ignore", invalid="ignore"):
            X = intr[v, 0] * pc[:, 0] / z + intr[v, 2]
            Y = intr[v, 1] * pc[:, 1] / z + intr[v, 3]
        ok = (z > near) & (X >= 0) & (X < wh[v, 0]) & (Y >= 0) & (Y < wh[v, 1])
        view[todo[ok]] = v[ok]
        todo = todo[~ok]
    out = x.copy()
    has = view >= 0
    c = centre[view[has]]
    d = x[has] - c
    out[has] = c + dist * d / np.linalg.norm(d, axis=1, keepdims=True)
    return out.astype(np.float32), view
