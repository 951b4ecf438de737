"""Outlier modes for the precision and stress workload.

A fraction of the stored leaf modes is replaced by points drawn uniformly in
the room volume, so that a matching share of pixel-to-mode correspondences
are outliers.  This prepares inputs only (both the library and the oracle
then read the same decoded mode positions); it holds none of the method's
arithmetic."""
from __future__ import annotations

import numpy as np


def replace_modes(mode_pos, nmodes, lo, hi, fraction=0.6, seed=13):
    """Returns a copy of mode_pos ([L][M][3]) in which each stored mode
    (rank < nmodes[leaf]) is, with probability `fraction`, moved to a point
    uniform in the box [lo, hi].  Draws come from numpy's PCG64 seeded with
    `seed`, one (u, x, y, z) quadruple per (leaf, rank) in row-major order,
    so the result does not depend on which modes are stored."""
    pos = np.array(mode_pos, dtype=np.float32, copy=True)
    L, M, _ = pos.shape
    rng = np.random.Generator(np.random.PCG64(seed))
    draws = rng.random((L, M, 4))
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    stored = np.arange(M)[None, :] < np.asarray(nmodes, np.int64)[:, None]
    hit = stored & (draws[:, :, 0] < fraction)
    pts = (lo + draws[:, :, 1:] * (hi - lo)).astype(np.float32)
    pos[hit] = pts[hit]
    return pos, hit
