"""Belief map and pose estimate (oracle).

Section III-A.3 (end): the belief tensor becomes a belief map by taking the maximum over
the channels for each cell, and the estimate is the most probable location.  The summed
marginal over channels is offered beside the paper's max.  Ties in the argmax go to the
lowest linear index of the [K][H][W] tensor.
"""
from __future__ import annotations

import numpy as np


def belief_map(b: np.ndarray, mode: str = "max") -> np.ndarray:
    """m[j][i] = max_k b[k][j][i] (paper) or sum_k b[k][j][i] (marginal)."""
    return b.max(axis=0) if mode == "max" else b.sum(axis=0)


def argmax_pose(b: np.ndarray):
    """(k, j, i, p) of the largest entry; the first in [K][H][W] order on ties."""
    flat = int(np.argmax(b.reshape(-1)))
    K, H, W = b.shape
    k, rem = divmod(flat, H * W)
    j, i = divmod(rem, W)
    return k, j, i, float(b[k, j, i])


def estimate(b: np.ndarray, cell: float, theta_t: float, radius_m: float, dk: int) -> dict:
    """The pose estimate and how concentrated the belief is around it (FP64).

    * The estimate is the argmax state (k, j, i) (``argmax_pose``): pose ((i + 1/2) c,
      (j + 1/2) c, 2 pi k / K + theta_t mod 2 pi), belief p.
    * mass_near: the belief within the disk of cells whose centres lie within radius_m of
      (j, i) -- dj^2 + di^2 <= floor(radius_m^2 / c^2 + 1e-9), the 1e-9 so that a radius of a
      whole number of cells includes the cells at that distance -- and within dk bins of k
      (circular).
    * The second hypothesis: the largest belief-map value (max over bins) among the cells
      outside that disk, the lowest cell index on ties; (-1, -1, 0) when none holds belief.
      second_ratio = its value / p.
    """
    K, H, W = b.shape
    k, j, i, p = argmax_pose(b)
    r2 = int(np.floor(radius_m * radius_m / (cell * cell) + 1e-9))
    J, I = np.mgrid[0:H, 0:W]
    inside = (J - j) ** 2 + (I - i) ** 2 <= r2
    kk = np.arange(K)
    dkk = np.minimum(np.abs(kk - k), K - np.abs(kk - k))
    near = (dkk <= dk)[:, None, None] & inside[None]
    m = b.max(axis=0)
    outside = np.where(inside, -1.0, m)
    flat = int(np.argmax(outside.reshape(-1)))
    v2 = float(outside.reshape(-1)[flat])
    if v2 > 0.0:
        sj, si = divmod(flat, W)
    else:
        sj, si, v2 = -1, -1, 0.0
    return dict(k=k, j=j, i=i, x=(i + 0.5) * cell, y=(j + 0.5) * cell,
                theta=(2.0 * np.pi * k / K + theta_t) % (2.0 * np.pi), p=p,
                mass_near=float(b[near].sum()), second_j=sj, second_i=si, second_p=v2,
                second_ratio=v2 / p if p > 0 else 0.0)
