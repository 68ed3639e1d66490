"""Seeded random walk of the ground-truth pose on free space, and the odometry it produces.

Poses are (x, y, heading) in metres / radians in the map frame; cell (j, i) covers
[i*c, (i+1)*c) x [j*c, (j+1)*c).  The odometry of one step is the relative pose between
consecutive ground-truth poses, expressed in the robot frame at the earlier pose:
(u, v) = forward / left translation, w = heading change.  Noise: each translation
component gets N(0, (frac * |(u, v)|)^2) and w gets N(0, rot_sigma^2).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass
class Walk:
    poses: np.ndarray       # (n+1, 3) ground-truth (x, y, heading)
    odom_true: np.ndarray   # (n, 3) exact relative poses (u, v, w)
    odom: np.ndarray        # (n, 3) noisy relative poses


def _free_at(occ: np.ndarray, cell: float, x: float, y: float, clearance: float) -> bool:
    H, W = occ.shape
    r = int(math.ceil(clearance / cell))
    i, j = int(math.floor(x / cell)), int(math.floor(y / cell))
    if i - r < 0 or j - r < 0 or i + r >= W or j + r >= H:
        return False
    return not occ[j - r:j + r + 1, i - r:i + r + 1].any()


def random_walk(occ: np.ndarray, cell: float, n_steps: int, dt: float, seed: int,
                speed=(0.3, 0.6), yaw_rate=(-0.5, 0.5), redraw_s: float = 1.0,
                trans_noise_frac: float = 0.02, rot_sigma: float = 0.01,
                clearance: float | None = None, start=None) -> Walk:
    """Ground-truth random walk plus noisy relative-pose odometry.

    Speed and yaw rate are redrawn every `redraw_s` seconds.  A step whose end point has an
    occupied cell within `clearance` (default one cell) is redrawn (up to 20 tries), else the
    robot turns in place.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    if clearance is None:
        clearance = cell
    free = np.argwhere(occ == 0)
    if start is None:
        for _ in range(10000):
            j, i = free[int(rng.integers(len(free)))]
            x, y = (i + 0.5) * cell, (j + 0.5) * cell
            if _free_at(occ, cell, x, y, clearance):
                break
        th = float(rng.uniform(-math.pi, math.pi))
    else:
        x, y, th = start
    v = float(rng.uniform(*speed))
    om = float(rng.uniform(*yaw_rate))
    per = max(1, int(round(redraw_s / dt)))
    poses = [(x, y, th)]
    rel = []
    for s in range(n_steps):
        if s % per == 0 and s > 0:
            v = float(rng.uniform(*speed))
            om = float(rng.uniform(*yaw_rate))
        d, w = v * dt, om * dt
        ok = False
        for _ in range(20):
            nx, ny = x + d * math.cos(th), y + d * math.sin(th)
            if _free_at(occ, cell, nx, ny, clearance):
                ok = True
                break
            v = float(rng.uniform(*speed))
            om = float(rng.uniform(*yaw_rate))
            d, w = v * dt, om * dt
        if not ok:
            d = 0.0
            w = (abs(om) if om != 0 else 0.5) * dt
            nx, ny = x, y
        rel.append((d, 0.0, w))
        x, y, th = nx, ny, th + w
        poses.append((x, y, th))
    rel = np.asarray(rel, np.float64)
    noisy = rel.copy()
    tr = np.hypot(rel[:, 0], rel[:, 1])
    noisy[:, 0] += rng.normal(0.0, 1.0, len(rel)) * trans_noise_frac * tr
    noisy[:, 1] += rng.normal(0.0, 1.0, len(rel)) * trans_noise_frac * tr
    noisy[:, 2] += rng.normal(0.0, rot_sigma, len(rel))
    return Walk(np.asarray(poses, np.float64), rel, noisy)


def random_odometry(n: int, seed: int, trans_m=(0.0, 0.05), rot=(-0.05, 0.05)) -> np.ndarray:
    """Free-standing relative-pose messages (u, v, w) for stage tests (no map needed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    d = rng.uniform(*trans_m, n)
    a = rng.uniform(-math.pi, math.pi, n)
    return np.stack([d * np.cos(a), d * np.sin(a), rng.uniform(*rot, n)], axis=1)
