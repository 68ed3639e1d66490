"""Simulated 2-D LIDAR scans from a continuous ground-truth pose.

The world model is the occupancy grid itself (each occupied cell a solid square; the grid
boundary a wall).  True ranges come from a brute-force fine ray march (step `march` cells,
default 1/64) from the continuous pose, which is independent of any grid-traversal
algorithm.  Then Gaussian range noise is added, ranges are clipped to [0, r_max], and a
random fraction of beams drops out to r_max.
"""
from __future__ import annotations

import math

import numpy as np


def true_ranges(occ: np.ndarray, cell: float, pose, angles: np.ndarray, r_max: float,
                march: float = 1.0 / 64) -> np.ndarray:
    """Distance (m) along each beam from (x, y) to the first occupied cell or the grid edge,
    capped at r_max.  `angles` are relative to the heading."""
    H, W = occ.shape
    x, y, th = pose
    a = th + np.asarray(angles, np.float64)
    dx, dy = np.cos(a), np.sin(a)
    n = int(math.ceil(r_max / cell / march)) + 1
    ts = np.arange(1, n + 1) * march                      # in cells
    px = x / cell + np.outer(dx, ts)
    py = y / cell + np.outer(dy, ts)
    ii, jj = np.floor(px).astype(np.int64), np.floor(py).astype(np.int64)
    outside = (ii < 0) | (jj < 0) | (ii >= W) | (jj >= H)
    hit = outside.copy()
    inside = ~outside
    hit[inside] = occ[jj[inside], ii[inside]] != 0
    first = np.where(hit.any(axis=1), hit.argmax(axis=1), n - 1)
    r = ts[first] * cell
    return np.minimum(r, r_max)


def simulate_scan(occ: np.ndarray, cell: float, pose, seed: int, n_beams: int = 360,
                  angle_min: float = 0.0, angle_inc: float = math.pi / 180, r_max: float = 10.0,
                  noise_sigma: float = 0.05, dropout: float = 0.05,
                  march: float = 1.0 / 64) -> np.ndarray:
    """One noisy scan (float32 ranges, metres) from `pose` = (x, y, heading).  A coarser
    `march` (in cells) trades range accuracy (error below one march step) for speed."""
    rng = np.random.Generator(np.random.PCG64(seed))
    angles = angle_min + angle_inc * np.arange(n_beams)
    r = true_ranges(occ, cell, pose, angles, r_max, march=march)
    r = r + rng.normal(0.0, noise_sigma, n_beams)
    r = np.clip(r, 0.0, r_max)
    r[rng.random(n_beams) < dropout] = r_max
    return r.astype(np.float32)
