"""Seeded synthetic inputs: Gaussian scenes, pinhole cameras and camera paths.

This module only draws random numbers and builds camera matrices. It holds
none of the rasterizer's arithmetic (no projection, no covariance, no SH
evaluation, no blending), so both the CUDA path and the FP64 oracle can be
fed from it without sharing any of the method's code.

The paper renders Gaussian maps of real scenes (GS-SLAM exports, Sec. 5.1)
that are not available here; the scenes below are stand-ins with the shapes,
sizes and density structure of the workloads the rasterizer is measured on:

* ``uniform_box``     — 10k Gaussians uniform in a box in front of the camera,
                        SH degree 0 (256x256 image).
* ``clustered``       — N Gaussians, 90 % in 200 isotropic clusters (cluster
                        sigma log-uniform in [0.05, 1] m) and 10 % uniform in
                        a 20 m box, SH degree 3, camera inside the scene
                        (1920x1080 image).
* ``imbalance``       — clustered scene with 20 % of the Gaussians packed into
                        a narrow cone of the first view and 1 % large splats.

All arrays are float32, C-contiguous, structure-of-arrays:
means (N,3), log_scales (N,3), quats (N,4) as (w,x,y,z), opacity_logits (N,),
sh (N,(d+1)^2,3).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Degree-0 SH coefficient range that maps to RGB in [0, 1] under the real
# orthonormal basis (Y_00 = 1/(2 sqrt(pi))) with the usual +0.5 offset:
# rgb = Y_00 * c + 0.5  <=>  c = (rgb - 0.5) * 2 sqrt(pi).
_SH0_HALF_RANGE = math.sqrt(math.pi)


@dataclass
class Scene:
    means: np.ndarray
    log_scales: np.ndarray
    quats: np.ndarray
    opacity_logits: np.ndarray
    sh: np.ndarray
    sh_degree: int
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def subset(self, idx) -> "Scene":
        return Scene(self.means[idx].copy(), self.log_scales[idx].copy(),
                     self.quats[idx].copy(), self.opacity_logits[idx].copy(),
                     self.sh[idx].copy(), self.sh_degree, self.name)

    def arrays(self):
        return dict(means=self.means, log_scales=self.log_scales, quats=self.quats,
                    opacity_logits=self.opacity_logits, sh=self.sh)


@dataclass
class Camera:
    """Pinhole camera. ``world_to_cam`` is the 3x4 row-major [R|t] matrix.

    Camera frame: x right, y down, z forward (the image plane is z > 0).
    Pixel (i, j) covers [i, i+1) x [j, j+1); its centre is (i+0.5, j+0.5).
    """
    world_to_cam: np.ndarray  # (3, 4) float32
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    near_z: float = 0.2
    meta: dict = field(default_factory=dict)

    def flat(self) -> np.ndarray:
        return np.ascontiguousarray(self.world_to_cam, dtype=np.float32).reshape(12)


def _unit_quats(rng, n):
    q = rng.standard_normal((n, 4)).astype(np.float64)
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q.astype(np.float32)


def pinhole(width: int, height: int, fov_x_deg: float = 60.0,
            world_to_cam: np.ndarray | None = None, near_z: float = 0.2) -> Camera:
    """Camera with horizontal field of view ``fov_x_deg``, square pixels and
    the principal point at the image centre."""
    fx = (width / 2.0) / math.tan(math.radians(fov_x_deg) / 2.0)
    if world_to_cam is None:
        world_to_cam = np.concatenate([np.eye(3), np.zeros((3, 1))], axis=1)
    return Camera(np.asarray(world_to_cam, dtype=np.float32).reshape(3, 4),
                  float(np.float32(fx)), float(np.float32(fx)),
                  width / 2.0, height / 2.0, int(width), int(height), near_z,
                  meta={"fov_x_deg": fov_x_deg})


def look_at(position, forward) -> np.ndarray:
    """World-to-camera [R|t] for a camera at ``position`` looking along
    ``forward`` with world -y as 'up' (so the identity camera looks along +z
    with y down)."""
    c = np.asarray(position, dtype=np.float64)
    z = np.asarray(forward, dtype=np.float64)
    z = z / np.linalg.norm(z)
    down = np.array([0.0, 1.0, 0.0])
    x = np.cross(down, z)
    if np.linalg.norm(x) < 1e-8:
        x = np.cross(np.array([0.0, 0.0, 1.0]), z)
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    R = np.stack([x, y, z])
    t = -R @ c
    return np.concatenate([R, t[:, None]], axis=1).astype(np.float32)


# --------------------------------------------------------------------------
# Scenes
# --------------------------------------------------------------------------

def uniform_box(n: int = 10_000, seed: int = 0) -> Scene:
    """Means x,y ~ U[-2,2], z ~ U[2,8]; log-scales N(-3, 0.5); uniform random
    unit quaternions; opacity = sigmoid(N(0,1)); SH degree 0 with RGB ~ U[0,1]."""
    rng = np.random.default_rng(seed)
    means = np.empty((n, 3), np.float32)
    means[:, 0:2] = rng.uniform(-2.0, 2.0, (n, 2))
    means[:, 2] = rng.uniform(2.0, 8.0, n)
    log_scales = rng.normal(-3.0, 0.5, (n, 3)).astype(np.float32)
    quats = _unit_quats(rng, n)
    logits = rng.normal(0.0, 1.0, n).astype(np.float32)
    sh = rng.uniform(-_SH0_HALF_RANGE, _SH0_HALF_RANGE, (n, 1, 3)).astype(np.float32)
    return Scene(means, log_scales, quats, logits, sh, 0, f"uniform_box_n{n}_s{seed}")


def clustered(n: int = 1_000_000, seed: int = 1, n_clusters: int = 200,
              box: float = 10.0, background_frac: float = 0.10,
              sh_degree: int = 3) -> Scene:
    """Non-uniform density: (1-background_frac) of the means from a mixture of
    isotropic clusters (centres U over the box, sigma log-uniform [0.05, 1] m,
    equal weights), the rest uniform over the [-box, box]^3 box.
    Log-scales N(-4, 0.7); SH coefficients N(0, 0.2)."""
    rng = np.random.default_rng(seed)
    centres = rng.uniform(-box, box, (n_clusters, 3))
    sigmas = np.exp(rng.uniform(math.log(0.05), math.log(1.0), n_clusters))
    n_bg = int(round(n * background_frac))
    n_cl = n - n_bg
    which = rng.integers(0, n_clusters, n_cl)
    means = np.empty((n, 3), np.float64)
    means[:n_cl] = centres[which] + rng.standard_normal((n_cl, 3)) * sigmas[which, None]
    means[n_cl:] = rng.uniform(-box, box, (n_bg, 3))
    perm = rng.permutation(n)
    means = means[perm].astype(np.float32)
    log_scales = rng.normal(-4.0, 0.7, (n, 3)).astype(np.float32)
    quats = _unit_quats(rng, n)
    logits = rng.normal(0.0, 1.0, n).astype(np.float32)
    k = (sh_degree + 1) ** 2
    sh = rng.normal(0.0, 0.2, (n, k, 3)).astype(np.float32)
    return Scene(means, log_scales, quats, logits, sh, sh_degree,
                 f"clustered_n{n}_s{seed}")


def imbalance(n: int = 6_000_000, seed: int = 4, width: int = 3840, height: int = 2160,
              fov_x_deg: float = 60.0, packed_frac: float = 0.20,
              packed_screen_frac: float = 0.02, large_frac: float = 0.01) -> Scene:
    """Imbalance stress: a clustered scene where ``packed_frac`` of the
    Gaussians sit in a narrow cone around the first view's optical axis whose
    cross-section covers ``packed_screen_frac`` of that view's image area, and
    ``large_frac`` are large splats whose world sigma makes the projected
    3-sigma radius exceed 256 px at their depth in the first view."""
    base = clustered(n, seed)
    rng = np.random.default_rng(seed + 1000)
    n_pack = int(n * packed_frac)
    n_large = int(n * large_frac)
    idx = rng.permutation(n)
    pack, large = idx[:n_pack], idx[n_pack:n_pack + n_large]
    f = (width / 2.0) / math.tan(math.radians(fov_x_deg) / 2.0)
    plane_area = (width / f) * (height / f)          # image area at z = 1
    tan_half = math.sqrt(packed_screen_frac * plane_area / math.pi)
    depth = rng.uniform(2.0, 10.0, n_pack)
    ang = rng.uniform(0, 2 * math.pi, n_pack)
    rad = np.sqrt(rng.uniform(0, 1, n_pack)) * tan_half
    base.means[pack, 0] = (rad * np.cos(ang) * depth).astype(np.float32)
    base.means[pack, 1] = (rad * np.sin(ang) * depth).astype(np.float32)
    base.means[pack, 2] = depth.astype(np.float32)
    z = np.abs(base.means[large, 2]) + 0.5
    sigma = 256.0 * z / (3.0 * f) * rng.uniform(1.0, 2.0, n_large)
    base.log_scales[large] = np.log(sigma)[:, None].astype(np.float32)
    base.name = f"imbalance_n{n}_s{seed}"
    return base


# --------------------------------------------------------------------------
# Camera paths
# --------------------------------------------------------------------------

def _catmull_rom(p0, p1, p2, p3, t):
    t2, t3 = t * t, t * t * t
    pos = 0.5 * ((2 * p1) + (-p0 + p2) * t + (2 * p0 - 5 * p1 + 4 * p2 - p3) * t2
                 + (-p0 + 3 * p1 - 3 * p2 + p3) * t3)
    tan = 0.5 * ((-p0 + p2) + 2 * (2 * p0 - 5 * p1 + 4 * p2 - p3) * t
                 + 3 * (-p0 + 3 * p1 - 3 * p2 + p3) * t2)
    return pos, tan


def trajectory(n_views: int = 64, seed: int = 1003, radius: float = 4.0,
               n_waypoints: int = 8, sizes=((1280, 720), (640, 480)),
               fov_x_deg: float = 60.0) -> list[Camera]:
    """Smooth seeded camera path: a closed Catmull-Rom spline through
    ``n_waypoints`` points within ``radius`` of the origin, the camera looking
    along the tangent; view i uses ``sizes[i % len(sizes)]``."""
    rng = np.random.default_rng(seed)
    d = rng.standard_normal((n_waypoints, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    wp = d * radius * np.cbrt(rng.uniform(0.2, 1.0, (n_waypoints, 1)))
    cams = []
    for i in range(n_views):
        s = i * n_waypoints / n_views
        k = int(s)
        t = s - k
        pts = [wp[(k + j - 1) % n_waypoints] for j in range(4)]
        pos, tan = _catmull_rom(*pts, t)
        w, h = sizes[i % len(sizes)]
        cams.append(pinhole(w, h, fov_x_deg, look_at(pos, tan)))
    return cams


def random_poses(n_views: int, seed: int, radius: float = 2.0,
                 sizes=((3840, 2160),), fov_x_deg: float = 60.0,
                 first_identity: bool = True) -> list[Camera]:
    """Seeded camera poses near the origin looking roughly along +z."""
    rng = np.random.default_rng(seed)
    cams = []
    for i in range(n_views):
        w, h = sizes[i % len(sizes)]
        if first_identity and i == 0:
            cams.append(pinhole(w, h, fov_x_deg))
            continue
        pos = rng.uniform(-radius, radius, 3) * np.array([1.0, 1.0, 0.25])
        fwd = np.array([0.0, 0.0, 1.0]) + rng.normal(0, 0.15, 3)
        cams.append(pinhole(w, h, fov_x_deg, look_at(pos, fwd)))
    return cams


def _rot_y(deg: float) -> np.ndarray:
    a = math.radians(deg)
    return np.array([[math.cos(a), 0.0, math.sin(a)], [0.0, 1.0, 0.0], [-math.sin(a), 0.0, math.cos(a)]])


def motion(kind: str, n_frames: int, width: int = 1920, height: int = 1080, step: float | None = None,
           seed: int = 1005, fov_x_deg: float = 60.0) -> list[Camera]:
    """Camera motions of the paper's churn experiment (Sec. 5.4), starting
    from the identity camera (at the origin, looking +z):
      'orbit'     about a target 4 m ahead, ``step`` degrees per frame (0.5);
      'translate' sideways along +x, ``step`` metres per frame (0.01);
      'rotate'    in place about the vertical axis, ``step`` degrees per frame (1);
      'teleport'  an independent seeded pose every frame;
      'static'    the same pose every frame."""
    cams = []
    rng = np.random.default_rng(seed)
    target = np.array([0.0, 0.0, 4.0])
    for f in range(n_frames):
        if kind == "static":
            w2c = look_at([0.0, 0.0, 0.0], [0.0, 0.0, 1.0])
        elif kind == "orbit":
            rot = _rot_y((0.5 if step is None else step) * f)
            pos = target + rot @ np.array([0.0, 0.0, -4.0])
            w2c = look_at(pos, target - pos)
        elif kind == "translate":
            w2c = look_at([(0.01 if step is None else step) * f, 0.0, 0.0], [0.0, 0.0, 1.0])
        elif kind == "rotate":
            w2c = look_at([0.0, 0.0, 0.0], _rot_y((1.0 if step is None else step) * f) @ np.array([0.0, 0.0, 1.0]))
        elif kind == "teleport":
            pos = rng.uniform(-2.0, 2.0, 3)
            fwd = rng.standard_normal(3)
            w2c = look_at(pos, fwd)
        else:
            raise KeyError(kind)
        cams.append(pinhole(width, height, fov_x_deg, w2c))
    return cams


def l1_target(height: int, width: int, seed: int) -> np.ndarray:
    """Seeded random target image, U[0,1], HWC float32."""
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, 1.0, (height, width, 3)).astype(np.float32)


# --------------------------------------------------------------------------
# Named workloads
# --------------------------------------------------------------------------

def workload(name: str):
    """(scene, cameras) for a named workload."""
    if name == "uniform_box_256":
        return uniform_box(10_000, 0), [pinhole(256, 256, 60.0)]
    if name == "clustered_1m_1080p":
        return clustered(1_000_000, 1), [pinhole(1920, 1080, 60.0)]
    if name == "clustered_500k_1080p":
        return clustered(500_000, 2), [pinhole(1920, 1080, 60.0)]
    if name == "clustered_1m_traj64":
        return clustered(1_000_000, 3), trajectory(64, 1003)
    if name == "imbalance_6m_4k_x8":
        return imbalance(6_000_000, 4), random_poses(8, 1004)
    if name == "imbalance_1m_4k_x2":
        return imbalance(1_000_000, 4), random_poses(2, 1004)
    raise KeyError(name)
