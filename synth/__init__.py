"""Seeded synthetic RGB-D workloads (rooms, trajectories, query frames).

This package only manufactures inputs.  It holds none of the relocaliser's
arithmetic: it renders an analytic textured room from given poses, draws
camera trajectories and query poses, and corrupts depth.  Both the CUDA path
and the CPU oracle consume what it produces; neither is imported here.
"""
from .rooms import (  # noqa: F401
    Room, Intrinsics, render, training_trajectory, query_poses,
    look_pose, mask_depth, noisy_depth, subsample, intrinsics_for,
)
