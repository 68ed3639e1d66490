"""Odometry bookkeeping (oracle, FP64).

Section III-A: a state [i, j, k] means pose (i*dW, j*dH, k*dTheta + theta_t); the internal
orientation offset advances as theta_t = theta_{t-1} + w for each motion update
u_t = {u, v, w}.  Eq. 2: the motion of channel k is the odometry translation rotated by that
channel's orientation.  Alg. 1 (its gate): the channels are propagated only when
|u_{t,k}| >= 1 (in cells).

Reading used here (the paper leaves the frame of (u, v) implicit): (u, v, w) is the
relative pose between consecutive robot poses, (u, v) in the robot frame at t-1.  A
hypothesis in channel k has heading k*dTheta + theta_{t-1}, so it moves by
R(k*dTheta) R(theta_{t-1}) [u, v]^T in the map frame.  Translations accumulate in
p = sum R(theta_{s-1}) [u_s, v_s]^T until the gate opens; channel k is then shifted by
R(k*dTheta) p / cell (cells), and p is cleared.
"""
from __future__ import annotations

import math

import numpy as np


def rot(a: float) -> np.ndarray:
    return np.array([[math.cos(a), -math.sin(a)], [math.sin(a), math.cos(a)]])


class Odometry:
    def __init__(self, K: int, cell: float, min_shift_cells: float = 0.0):
        self.K = K
        self.cell = cell
        self.min_shift = min_shift_cells
        self.theta = 0.0
        self.p = np.zeros(2)

    def add(self, u: float, v: float, w: float) -> None:
        """Accumulate one relative-pose message (Section III-A, Eq. 2)."""
        self.p = self.p + rot(self.theta) @ np.array([u, v])
        self.theta = self.theta + w

    def due(self) -> bool:
        """Alg. 1 gate |u_{t,k}| >= min_shift (cells); |R p| = |p| for every channel."""
        return math.hypot(self.p[0], self.p[1]) / self.cell >= self.min_shift

    def shifts(self) -> np.ndarray:
        """Eq. 2: per-channel displacement in cells, shape (K, 2) as (sx, sy)."""
        out = np.empty((self.K, 2))
        for k in range(self.K):
            out[k] = rot(2.0 * math.pi * k / self.K) @ self.p / self.cell
        return out

    def consume(self) -> None:
        self.p = np.zeros(2)
