"""Seeded workload recipes (rooms, forests, training trajectories, queries).

Each recipe lists every parameter a run needs, as plain values: the room,
the resolution, the forest and relocaliser settings and the seeds.  The
relocaliser parameter names follow the paper's parameter table; values the
paper leaves open are this library's readings.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from .rooms import Room, intrinsics_for, mask_depth, noisy_depth, query_poses, render, training_trajectory

# Default relocaliser of the paper's parameter table (Appendix B) with the
# open values filled in.
RANSAC_DEFAULT = dict(
    n_hyp=1024, max_iter=6000, n_cull=64, eta=512, k_out=16, pose_update=1, use_cov=1,
    colour_thresh=30, min_sq_dist=0.09, max_trans_err=0.05, k_top=10, n_trees_used=5,
    lm_max_iter=10, batch_attempts=32, lm_lambda0=1e-3, lm_inlier_thresh=0.1, lm_stop=1e-6,
    rank=1, halve_to_one=0,
)
# ICP before ranking (Sec. 3.2.4, the library's reading R21), switched on.
ICP_ON = dict(icp=1, icp_levels=3, icp_stride=(4, 2, 1), icp_iters=(6, 3, 2),
              icp_dist=(0.1, 0.05, 0.025), icp_min_frac=0.5, icp_ridge=1e-4)
FOREST_DEFAULT = dict(
    n_trees=5, depth=15, p_depth=0.4, delta_lo=-130.0, delta_hi=130.0, tau_depth_lo=-0.2,
    tau_depth_hi=0.2, tau_rgb_lo=-50.0, tau_rgb_hi=50.0, tau_zero=0, kappa=1024, m_max=50,
    min_cluster_size=20, sigma=0.1, tau_c=0.05, cov_eps=1e-4, mode_precision=1, grid_step=4,
    grid_origin=0,
)


@dataclasses.dataclass
class Workload:
    name: str
    room_size: tuple
    room_seed: int
    width: int
    height: int
    forest: dict
    forest_seed: int
    n_train: int
    ransac: dict
    n_queries: int
    query_seed: int = 1000
    noise_sigma: float = 0.002

    @property
    def K(self):
        return intrinsics_for(self.width, self.height)

    def room(self):
        return Room(self.room_size, self.room_seed)

    def training_frames(self):
        """Yields (depth, rgb, cam_to_world) of the training trajectory."""
        room = self.room()
        for i, T in enumerate(training_trajectory(room, self.n_train)):
            d, c = render(room, self.K, T, self.noise_sigma, noise_seed=100 + i)
            yield d, c, T

    def query(self, q: int):
        """(depth, rgb, ground-truth pose, query seed) of query q."""
        room = self.room()
        T = query_poses(room, q + 1, seed=self.query_seed)[q]
        d, c = render(room, self.K, T, self.noise_sigma, noise_seed=5000 + q)
        return d, c, T, self.query_seed + q

    def queries(self, n=None):
        room = self.room()
        n = self.n_queries if n is None else n
        poses = query_poses(room, n, seed=self.query_seed)
        out = []
        for q, T in enumerate(poses):
            d, c = render(room, self.K, T, self.noise_sigma, noise_seed=5000 + q)
            out.append((d, c, T, self.query_seed + q))
        return out


# Config 1: single query, plain method, small room render and forest.
CONFIG1 = Workload(
    name="room4x3x2.5_160x120_1tree_d10", room_size=(4.0, 3.0, 2.5), room_seed=5,
    width=160, height=120,
    forest=dict(FOREST_DEFAULT, n_trees=1, depth=10, kappa=256, m_max=10, min_cluster_size=5),
    forest_seed=2, n_train=20,
    ransac=dict(RANSAC_DEFAULT, n_hyp=64, n_cull=64, eta=100, k_out=1, k_top=10, n_trees_used=1),
    n_queries=16,
)

# Config 2: paper-shaped single query at 640x480.
CONFIG2 = Workload(
    name="room4x3x2.5_640x480_5trees_d15", room_size=(4.0, 3.0, 2.5), room_seed=5,
    width=640, height=480,
    forest=dict(FOREST_DEFAULT),
    forest_seed=2, n_train=200,
    ransac=dict(RANSAC_DEFAULT, n_hyp=1024, n_cull=64, eta=500, k_out=16, halve_to_one=1),
    n_queries=16,
)

# Config 5: precision and stress on the config-2 room and forest training:
# 4096 hypotheses, every stored mode of a leaf used (K_top = M_max = 50),
# 60% of the stored modes replaced by outliers uniform in the room
# (synth.outliers, seed 13), FP16-offset vs FP32 mode storage, 200 queries.
CONFIG5_OUTLIER_FRACTION = 0.6
CONFIG5_OUTLIER_SEED = 13


def config5(mode_precision: int) -> Workload:
    """mode_precision: 1 = FP16 offsets from FP32 leaf centroids, 0 = FP32."""
    tag = "fp16" if mode_precision else "fp32"
    return Workload(
        name=f"room4x3x2.5_640x480_5trees_d15_outliers60_{tag}", room_size=(4.0, 3.0, 2.5), room_seed=5,
        width=640, height=480,
        forest=dict(FOREST_DEFAULT, mode_precision=mode_precision),
        forest_seed=2, n_train=200,
        ransac=dict(RANSAC_DEFAULT, n_hyp=4096, n_cull=64, eta=500, k_out=16, halve_to_one=1, k_top=50),
        n_queries=200,
    )


# Config 4: serving over three rooms, each with its own five-tree forest;
# 8 camera streams (room = stream mod 3; even streams 640x480, odd 320x240)
# with Poisson arrivals at 30 Hz per stream (seed 11 + stream).
SERVING_ROOMS = [
    CONFIG2,
    Workload(name="room6x5x3_640x480_5trees_d15", room_size=(6.0, 5.0, 3.0), room_seed=17,
             width=640, height=480, forest=dict(FOREST_DEFAULT), forest_seed=3, n_train=200,
             ransac=dict(CONFIG2.ransac), n_queries=16),
    Workload(name="room10x8x3_640x480_5trees_d15", room_size=(10.0, 8.0, 3.0), room_seed=29,
             width=640, height=480, forest=dict(FOREST_DEFAULT), forest_seed=4, n_train=200,
             ransac=dict(CONFIG2.ransac), n_queries=16),
]
SERVING_STREAMS = 8
SERVING_RATE_HZ = 30.0


def serving_arrivals(seconds: float, rate_scale: float = 1.0, streams: int = SERVING_STREAMS,
                     seed: int = 11):
    """Sorted (time in s, stream) of Poisson arrivals at SERVING_RATE_HZ x
    rate_scale per stream over [0, seconds)."""
    out = []
    for s in range(streams):
        rng = np.random.default_rng(seed + s)
        t = rng.exponential(1.0 / (SERVING_RATE_HZ * rate_scale))
        while t < seconds:
            out.append((t, s))
            t += rng.exponential(1.0 / (SERVING_RATE_HZ * rate_scale))
    out.sort()
    return out


# Robustness sweeps (missing and noisy depth; reading R22: the corruption is
# applied to every depth image, training frames and queries alike).
MISSING_LEVELS = (0.0, 0.1, 0.2, 0.3, 0.5, 0.7, 0.8, 0.9, 0.95)
NOISE_LEVELS = (0.0, 0.025, 0.05, 0.075, 0.1)
_CORRUPT_SEED = {"missing": 70000, "noise": 90000}


def corrupt(depth, kind: str, level: float, index: int):
    """Depth image `index` of a sweep corrupted at `level`: missing depth
    (zero iff r <= p, r ~ U[0,1] per pixel) or depth-dependent noise
    (d + n d, n ~ N(0, sigma^2) per pixel); training frames use indices
    0.., queries 10000 + q.  Level 0 returns the image unchanged."""
    if level == 0:
        return depth
    seed = _CORRUPT_SEED[kind] + index
    if kind == "missing":
        return mask_depth(depth, level, seed)
    if kind == "noise":
        return noisy_depth(depth, level, seed)
    raise ValueError(kind)


# Config 3 levels (shared config-2 forest): subsample, relocaliser parameters.
CASCADE_LEVELS = [
    (4, dict(RANSAC_DEFAULT, n_hyp=64, n_trees_used=1, k_out=1, eta=100)),
    (2, dict(RANSAC_DEFAULT, n_hyp=256, n_trees_used=5, k_out=1, eta=250)),
    (1, dict(RANSAC_DEFAULT, n_hyp=1024, n_trees_used=5, k_out=16, eta=500)),
]


def cascade_thresholds(seed: int = 7):
    """tau_1, tau_2 drawn uniformly from [0.04, 0.09] m (the paper tuned
    5 cm and 7.5 cm on its datasets)."""
    r = np.random.default_rng(seed).uniform(0.04, 0.09, size=2)
    return [float(r[0]), float(r[1])]


def small_case(n_trees=2, depth=8, width=96, height=72, n_train=12, **ransac):
    """A few-second oracle case that still spans several tiles, a ragged
    tail and multiple trees.  Its checks are loosened (colour 120, rigidity
    0.15 m, spread 0.2 m) so that most generation slots succeed and the
    cull, the rounds and LM all see many hypotheses."""
    return Workload(
        name=f"room4x3x2.5_{width}x{height}_{n_trees}trees_d{depth}", room_size=(4.0, 3.0, 2.5),
        room_seed=5, width=width, height=height,
        forest=dict(FOREST_DEFAULT, n_trees=n_trees, depth=depth, kappa=128, m_max=8,
                    min_cluster_size=3, tau_c=0.2),
        forest_seed=3, n_train=n_train,
        ransac=dict(RANSAC_DEFAULT, n_hyp=96, n_cull=24, eta=64, k_out=4, k_top=4,
                    n_trees_used=n_trees, max_iter=2000, colour_thresh=120, max_trans_err=0.15,
                    min_sq_dist=0.04, halve_to_one=1, **ransac),
        n_queries=4,
    )
