"""Seeded synthetic rooms standing in for the paper's indoor RGB-D datasets.

The paper evaluates on 640x480 Kinect-style registered RGB-D frames of
indoor scenes a few metres across (Sec. 4, 7-Scenes / Stanford 4 Scenes).
Those datasets are not available, so every workload here is an analytic
axis-aligned box room [0,X]x[0,Y]x[0,Z] (z up) whose six inner faces are
tiled with 8 cm square cells of seeded random colour.  Frames are rendered
by casting one ray per pixel from a pinhole camera (x right, y down,
z forward); depth is the z-depth of the first wall hit plus Gaussian noise,
colour is the colour of the hit cell (no lighting).

Random draws here use numpy's own generator; they are input synthesis only.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

CELL = 0.08  # metres, side of a texture cell


@dataclasses.dataclass(frozen=True)
class Intrinsics:
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int


def intrinsics_for(width: int, height: int) -> Intrinsics:
    """Kinect-like intrinsics used by the workloads (fx=585 at 640x480)."""
    if (width, height) == (160, 120):
        return Intrinsics(146.0, 146.0, 80.0, 60.0, 160, 120)
    scale = width / 640.0
    return Intrinsics(585.0 * scale, 585.0 * scale, 320.0 * scale, 240.0 * scale,
                      width, height)


@dataclasses.dataclass
class Room:
    """Axis-aligned textured box room."""
    size: tuple[float, float, float]
    seed: int

    def __post_init__(self):
        rng = np.random.default_rng(self.seed)
        X, Y, Z = self.size
        # face order: x=0, x=X, y=0, y=Y, z=0, z=Z; each face is indexed by
        # the two remaining axes in increasing axis order.
        dims = [(Y, Z), (Y, Z), (X, Z), (X, Z), (X, Y), (X, Y)]
        self.textures = []
        for a, b in dims:
            na, nb = int(math.ceil(a / CELL)) + 1, int(math.ceil(b / CELL)) + 1
            self.textures.append(rng.integers(0, 256, size=(na, nb, 3), dtype=np.uint8))

    @property
    def lo(self):
        return np.zeros(3)

    @property
    def hi(self):
        return np.asarray(self.size, dtype=np.float64)


def look_pose(position, yaw, pitch, roll=0.0) -> np.ndarray:
    """Camera->world 4x4 pose for a camera at `position` looking along
    (yaw, pitch) with world z up; camera axes x right, y down, z forward."""
    cp, sp = math.cos(pitch), math.sin(pitch)
    f = np.array([cp * math.cos(yaw), cp * math.sin(yaw), sp])
    up = np.array([0.0, 0.0, 1.0])
    r = np.cross(f, up)
    r /= np.linalg.norm(r)
    d = np.cross(f, r)
    R = np.stack([r, d, f], axis=1)
    if roll:
        c, s = math.cos(roll), math.sin(roll)
        R = R @ np.array([[c, -s, 0], [s, c, 0], [0, 0, 1.0]])
    T = np.eye(4)
    T[:3, :3] = R
    T[:3, 3] = position
    return T


def _rodrigues(axis, angle):
    axis = np.asarray(axis, dtype=np.float64)
    axis = axis / np.linalg.norm(axis)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + math.sin(angle) * K + (1 - math.cos(angle)) * (K @ K)


def render(room: Room, K: Intrinsics, cam_to_world: np.ndarray, noise_sigma: float = 0.002,
           noise_seed: int = 0):
    """Render (depth float32 [H,W] metres, rgb uint8 [H,W,3]) of `room`."""
    W, H = K.width, K.height
    u = np.arange(W, dtype=np.float64)
    v = np.arange(H, dtype=np.float64)
    uu, vv = np.meshgrid(u, v)
    dc = np.stack([(uu - K.cx) / K.fx, (vv - K.cy) / K.fy, np.ones_like(uu)], axis=-1)
    R = cam_to_world[:3, :3]
    o = cam_to_world[:3, 3]
    dw = dc @ R.T
    lo, hi = room.lo, room.hi
    with np.errstate(divide="ignore", invalid="ignore"):
        t1 = (lo - o) / dw
        t2 = (hi - o) / dw
    tfar_axis = np.where(dw > 0, t2, np.where(dw < 0, t1, np.inf))
    axis = np.argmin(tfar_axis, axis=-1)
    t = np.take_along_axis(tfar_axis, axis[..., None], axis=-1)[..., 0]
    side = np.take_along_axis(dw, axis[..., None], axis=-1)[..., 0] > 0
    face = axis * 2 + side.astype(np.int64)
    p = o + t[..., None] * dw
    rgb = np.zeros((H, W, 3), dtype=np.uint8)
    other = {0: (1, 2), 1: (0, 2), 2: (0, 1)}
    for f in range(6):
        m = face == f
        if not m.any():
            continue
        a, b = other[f // 2]
        tex = room.textures[f]
        ia = np.clip((p[..., a][m] / CELL).astype(np.int64), 0, tex.shape[0] - 1)
        ib = np.clip((p[..., b][m] / CELL).astype(np.int64), 0, tex.shape[1] - 1)
        rgb[m] = tex[ia, ib]
    depth = t
    if noise_sigma > 0:
        rng = np.random.default_rng(noise_seed)
        depth = depth + rng.normal(0.0, noise_sigma, size=depth.shape)
    depth = np.where(np.isfinite(depth) & (depth > 0), depth, 0.0)
    return depth.astype(np.float32), rgb


def training_trajectory(room: Room, n_frames: int, seed: int = 3):
    """Seeded training trajectory: ellipse around the room centre at 1.5 m
    (clamped to the room height), yaw sweeping 360 degrees, +-10 degree
    pitch sinusoid, +-2 cm / +-2 degree jitter."""
    rng = np.random.default_rng(seed)
    X, Y, Z = room.size
    c = np.array([X / 2, Y / 2, min(1.5, Z * 0.6)])
    poses = []
    for i in range(n_frames):
        a = 2 * math.pi * i / n_frames
        pos = c + np.array([0.3 * X * math.cos(a), 0.3 * Y * math.sin(a), 0.0])
        pos = pos + rng.uniform(-0.02, 0.02, size=3)
        yaw = a + math.radians(rng.uniform(-2, 2))
        pitch = math.radians(10.0 * math.sin(3 * a) + rng.uniform(-2, 2))
        poses.append(look_pose(pos, yaw, pitch))
    return poses


def query_poses(room: Room, n: int, seed: int = 1000, n_traj: int = 720,
                max_trans: float = 0.3, max_rot_deg: float = 20.0):
    """Query poses near the training trajectory: a random trajectory pose
    perturbed by a translation of at most `max_trans` and a rotation of at
    most `max_rot_deg`, kept at least 0.5 m inside the walls."""
    traj = training_trajectory(room, n_traj, seed=3)
    out = []
    lo = room.lo + 0.5
    hi = room.hi - 0.5
    for q in range(n):
        rng = np.random.default_rng(seed + q)
        T = traj[int(rng.integers(0, n_traj))].copy()
        dirv = rng.normal(size=3)
        dirv /= np.linalg.norm(dirv)
        T[:3, 3] = np.clip(T[:3, 3] + dirv * max_trans * rng.uniform() ** (1 / 3), lo, hi)
        axis = rng.normal(size=3)
        T[:3, :3] = _rodrigues(axis, math.radians(max_rot_deg) * rng.uniform()) @ T[:3, :3]
        out.append(T)
    return out


def mask_depth(depth: np.ndarray, p: float, seed: int) -> np.ndarray:
    """Missing-depth corruption of Sec. A.4: zero pixel i iff r_i <= p, r_i ~ U[0,1]."""
    r = np.random.default_rng(seed).uniform(0.0, 1.0, size=depth.shape)
    return np.where(r <= p, 0.0, depth).astype(np.float32)


def noisy_depth(depth: np.ndarray, sigma: float, seed: int) -> np.ndarray:
    """Depth-dependent noise of Sec. A.4: d <- d + n*d, n ~ N(0, sigma^2)."""
    n = np.random.default_rng(seed).normal(0.0, sigma, size=depth.shape)
    return np.where(depth > 0, depth + n * depth, 0.0).astype(np.float32)


def subsample(depth: np.ndarray, rgb: np.ndarray, K: Intrinsics, s: int):
    """Pixel (u', v') of the result is pixel (s*u', s*v') of the input; the
    intrinsics scale by 1/s so back-projection stays consistent."""
    d = np.ascontiguousarray(depth[::s, ::s])
    c = np.ascontiguousarray(rgb[::s, ::s])
    Ks = Intrinsics(K.fx / s, K.fy / s, K.cx / s, K.cy / s, d.shape[1], d.shape[0])
    return d, c, Ks
