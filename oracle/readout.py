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
