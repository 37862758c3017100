"""Seeded synthetic inputs: Gaussian maps, cameras and poses.

This module holds only random-number draws and containers.  It contains none
of the rasterizer's arithmetic, so that the CPU oracle and the CUDA path can
both be fed from it without sharing any of the method.

The paper's datasets (Multi-agent Replica, 7-Scenes; Sec. 4.1) are not
available, so these scenes stand in for them: room-scale indoor volumes whose
Gaussians concentrate on planar walls, seen by RGB-D cameras at 640x480 or
1200x680.  A Gaussian is the map primitive of Sec. 3.3: mean x, covariance
from log-scales and a (w, x, y, z) rotation quaternion, opacity (stored as a
logit) and colour.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass(frozen=True)
class Camera:
    """Pinhole intrinsics; pixel (x, y) has its centre at (x + 0.5, y + 0.5)."""

    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    z_near: float = 0.2
    max_dist: float = 0.0  # > 0: only Gaussians within this distance of the camera are candidates

    @property
    def npix(self) -> int:
        return self.width * self.height

    @property
    def tiles_x(self) -> int:
        return (self.width + 15) // 16

    @property
    def tiles_y(self) -> int:
        return (self.height + 15) // 16

    @property
    def n_tiles(self) -> int:
        return self.tiles_x * self.tiles_y


@dataclasses.dataclass
class Scene:
    """Structure-of-arrays Gaussian map (float32 unless built otherwise)."""

    mean: np.ndarray  # [N, 3]
    log_scale: np.ndarray  # [N, 3]
    quat: np.ndarray  # [N, 4]  (w, x, y, z), not necessarily normalised
    opacity_logit: np.ndarray  # [N]
    rgb: np.ndarray  # [N, 3]

    @property
    def n(self) -> int:
        return int(self.mean.shape[0])

    def astype(self, dtype) -> "Scene":
        return Scene(*(np.ascontiguousarray(a, dtype=dtype) for a in self.arrays()))

    def arrays(self):
        return (self.mean, self.log_scale, self.quat, self.opacity_logit, self.rgb)

    def subset(self, idx) -> "Scene":
        return Scene(*(np.ascontiguousarray(a[idx]) for a in self.arrays()))


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _attributes(rng, n):
    log_scale = rng.normal(-3.0, 0.3, size=(n, 3))
    q = rng.normal(0.0, 1.0, size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    logit = rng.normal(0.0, 1.0, size=n)
    rgb = rng.uniform(0.0, 1.0, size=(n, 3))
    return log_scale, q, logit, rgb


def scene_uniform(n: int, seed: int) -> Scene:
    """Means uniform in x, y in [-1, 1], z in [2, 4] (the small forward case)."""
    rng = np.random.default_rng(seed)
    mean = np.stack([rng.uniform(-1, 1, n), rng.uniform(-1, 1, n), rng.uniform(2, 4, n)], axis=1)
    ls, q, lo, c = _attributes(rng, n)
    return Scene(_f32(mean), _f32(ls), _f32(q), _f32(lo), _f32(c))


ROOM_HALF = (2.0, 1.5, 1.5)  # 4 x 3 x 3 m box centred at the origin


def scene_room(n: int, seed: int, half=ROOM_HALF, wall_sigma: float = 0.02) -> Scene:
    """Room-shaped map: each Gaussian picks one of the 6 walls with probability
    proportional to its area, lies uniformly on it and is offset N(0, sigma)
    along the wall normal."""
    rng = np.random.default_rng(seed)
    hx, hy, hz = half
    areas = np.array([4 * hy * hz] * 2 + [4 * hx * hz] * 2 + [4 * hx * hy] * 2)
    wall = rng.choice(6, size=n, p=areas / areas.sum())
    u = rng.uniform(-1.0, 1.0, size=(n, 3)) * np.array(half)
    off = rng.normal(0.0, wall_sigma, size=n)
    axis = wall // 2
    sign = np.where(wall % 2 == 0, -1.0, 1.0)
    mean = u.copy()
    mean[np.arange(n), axis] = sign * np.array(half)[axis] + off
    ls, q, lo, c = _attributes(rng, n)
    return Scene(_f32(mean), _f32(ls), _f32(q), _f32(lo), _f32(c))


def scene_wall_patch(n: int, seed: int, z: float = 1.5, extent=(0.45, 0.32)) -> Scene:
    """Small sub-scene: n Gaussians on a patch of the +z wall in front of an
    identity-pose camera (the finite-difference case)."""
    rng = np.random.default_rng(seed)
    mean = np.stack(
        [rng.uniform(-extent[0], extent[0], n), rng.uniform(-extent[1], extent[1], n),
         z + rng.normal(0.0, 0.02, n)], axis=1)
    ls, q, lo, c = _attributes(rng, n)
    return Scene(_f32(mean), _f32(ls), _f32(q), _f32(lo), _f32(c))


def identity_w2c() -> np.ndarray:
    return np.eye(4, dtype=np.float32)


def _rotation(axis, angle):
    axis = np.asarray(axis, dtype=np.float64)
    axis = axis / np.linalg.norm(axis)
    k = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + math.sin(angle) * k + (1 - math.cos(angle)) * (k @ k)


def perturbed_w2c(seed: int, trans_m: float = 0.01, rot_deg: float = 0.5, base=None) -> np.ndarray:
    """A pose displaced by `trans_m` metres along a random direction and
    rotated by `rot_deg` degrees about a random axis."""
    rng = np.random.default_rng(seed)
    d = rng.normal(size=3)
    d *= trans_m / np.linalg.norm(d)
    a = rng.normal(size=3)
    P = np.eye(4)
    P[:3, :3] = _rotation(a, math.radians(rot_deg))
    P[:3, 3] = d
    B = np.eye(4) if base is None else np.asarray(base, dtype=np.float64)
    return np.ascontiguousarray(P @ B, dtype=np.float32)


def look_at_w2c(eye, target, up=(0.0, -1.0, 0.0)) -> np.ndarray:
    """World-to-camera matrix of a camera at `eye` looking at `target`
    (camera x right, y down, z forward)."""
    eye = np.asarray(eye, dtype=np.float64)
    f = np.asarray(target, dtype=np.float64) - eye
    f /= np.linalg.norm(f)
    # camera x (right) = forward x up, with up = -y so that y points down
    r = np.cross(f, np.asarray(up, dtype=np.float64))
    r /= np.linalg.norm(r)
    d = np.cross(f, r)
    Rcw = np.stack([r, d, f])  # rows: camera axes in world
    w2c = np.eye(4)
    w2c[:3, :3] = Rcw
    w2c[:3, 3] = -Rcw @ eye
    return np.ascontiguousarray(w2c, dtype=np.float32)


# ---------------------------------------------------------------------------
# Named workloads (sizes from the paper-shaped configurations).
# ---------------------------------------------------------------------------
CAM_SMALL = Camera(128, 96, 100.0, 100.0, 64.0, 48.0)
CAM_VGA = Camera(640, 480, 525.0, 525.0, 320.0, 240.0)
CAM_WIDE = Camera(1200, 680, 600.0, 600.0, 600.0, 340.0)


def workload_small_forward(seed: int = 0):
    """2,000 Gaussians, identity pose, 128x96, black background."""
    return scene_uniform(2000, seed), identity_w2c(), CAM_SMALL, np.zeros(3, np.float32)


def workload_track_map(seed: int = 1, n: int = 300_000):
    """Single-agent tracking/mapping step: 300k-Gaussian room, 640x480,
    camera at the room centre looking at the +z wall; the target is rendered
    from a pose perturbed by 1 cm / 0.5 degrees."""
    scene = scene_room(n, seed)
    return scene, identity_w2c(), perturbed_w2c(seed + 1000), CAM_VGA, np.zeros(3, np.float32)


def workload_multi_agent(seed: int = 2, sizes=(150_000, 400_000, 900_000)):
    """Several agents of uneven map sizes, each a room scene at 1200x680."""
    seeds = [seed, 20, 21]
    out = []
    for i, n in enumerate(sizes):
        s = scene_room(n, seeds[i % len(seeds)] + 100 * (i // len(seeds)))
        out.append((s, perturbed_w2c(seeds[i % len(seeds)] + 500, 0.05, 3.0), CAM_WIDE))
    return out


def keyframe_poses(n_views: int = 8, seed: int = 3):
    """Overlapping keyframe poses along a short path inside the room, all
    looking roughly at the +z wall."""
    rng = np.random.default_rng(seed)
    poses = []
    for k in range(n_views):
        t = k / max(1, n_views - 1)
        eye = np.array([-0.6 + 1.2 * t, 0.1 * math.sin(3 * t), -0.3 + 0.2 * t])
        target = np.array([0.4 * (t - 0.5), 0.0, 1.5]) + rng.normal(0, 0.05, 3)
        poses.append(look_at_w2c(eye, target))
    return poses


def serving_agents(seed: int = 4, n_agents: int = 8, lo: int = 100_000, hi: int = 2_000_000):
    """Agents with map sizes log-uniform in [lo, hi]; agents 0-3 at 640x480,
    4-7 at 1200x680."""
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(math.log(lo), math.log(hi), n_agents)).astype(np.int64)
    agents = []
    for a in range(n_agents):
        cam = CAM_VGA if a < n_agents // 2 else CAM_WIDE
        agents.append(dict(n=int(sizes[a]), seed=1000 + a, cam=cam))
    return agents


def _quat_of_rotation(R):
    """(w, x, y, z) unit quaternion of a rotation matrix (Shepperd's method)."""
    R = np.asarray(R, dtype=np.float64)
    tr = np.trace(R)
    if tr > 0:
        s = 2.0 * math.sqrt(1.0 + tr)
        return np.array([0.25 * s, (R[2, 1] - R[1, 2]) / s, (R[0, 2] - R[2, 0]) / s, (R[1, 0] - R[0, 1]) / s])
    i = int(np.argmax(np.diag(R)))
    j, k = (i + 1) % 3, (i + 2) % 3
    s = 2.0 * math.sqrt(1.0 + R[i, i] - R[j, j] - R[k, k])
    q = np.zeros(4)
    q[0] = (R[k, j] - R[j, k]) / s
    q[1 + i] = 0.25 * s
    q[1 + j] = (R[j, i] + R[i, j]) / s
    q[1 + k] = (R[k, i] + R[i, k]) / s
    return q


def transform_scene(scene: Scene, T) -> Scene:
    """The scene moved rigidly by T (4x4): means x -> R x + t, rotations
    q -> q_R * q (Hamilton product); scales, opacities and colours unchanged."""
    T = np.asarray(T, dtype=np.float64)
    R, t = T[:3, :3], T[:3, 3]
    mean = scene.mean.astype(np.float64) @ R.T + t
    a = _quat_of_rotation(R)
    q = scene.quat.astype(np.float64)
    w = a[0] * q[:, 0] - a[1] * q[:, 1] - a[2] * q[:, 2] - a[3] * q[:, 3]
    x = a[0] * q[:, 1] + a[1] * q[:, 0] + a[2] * q[:, 3] - a[3] * q[:, 2]
    y = a[0] * q[:, 2] - a[1] * q[:, 3] + a[2] * q[:, 0] + a[3] * q[:, 1]
    z = a[0] * q[:, 3] + a[1] * q[:, 2] - a[2] * q[:, 1] + a[3] * q[:, 0]
    return Scene(_f32(mean), scene.log_scale.copy(), _f32(np.stack([w, x, y, z], 1)), scene.opacity_logit.copy(),
                 scene.rgb.copy())


def workload_alignment(seed: int = 3, n: int = 1_000_000, n_views: int = 8, cam: Camera = CAM_WIDE):
    """Two agents that mapped the same room: A's map, and B's map of the same
    surfaces (A's Gaussians in a shuffled order, means jittered by 2 mm and
    colours by 0.02) held in B's own world frame, which differs from A's by
    T_true (B world -> A world: 20 cm and 10 degrees).  Returns A's map, B's
    map, T_true, A's keyframe poses and the alignment's starting transform,
    T_true perturbed by 1 cm / 0.5 degrees."""
    a = scene_room(n, seed)
    rng = np.random.default_rng(seed + 77)
    perm = rng.permutation(n)
    b = a.subset(perm)
    b.mean = _f32(b.mean + rng.normal(0.0, 0.002, b.mean.shape))
    b.rgb = _f32(np.clip(b.rgb + rng.normal(0.0, 0.02, b.rgb.shape), 0.0, 1.0))
    T_true = perturbed_w2c(seed + 200, 0.2, 10.0).astype(np.float64)
    b = transform_scene(b, np.linalg.inv(T_true))
    T0 = perturbed_w2c(seed + 300, 0.01, 0.5, base=T_true)
    return a, b, perm, T_true.astype(np.float32), keyframe_poses(n_views, seed), T0, cam
