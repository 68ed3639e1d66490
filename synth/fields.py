"""Seeded random fields for stage tests: belief-like tensors and belief maps.

Values are non-negative, zero on occupied cells, with a mix of smooth structure and a few
sharp peaks, so that tests exercise both flat regions and large dynamic range.
"""
from __future__ import annotations

import numpy as np


def belief_like(occ: np.ndarray, K: int, seed: int, peaks: int = 8,
                dtype=np.float64) -> np.ndarray:
    """A [K][H][W] non-negative field, zero where occ != 0, summing to 1."""
    rng = np.random.Generator(np.random.PCG64(seed))
    H, W = occ.shape
    b = rng.random((K, H, W)) ** 4
    for _ in range(peaks):
        k, j, i = int(rng.integers(K)), int(rng.integers(H)), int(rng.integers(W))
        b[k, j, i] += float(rng.uniform(50, 500))
    b *= (occ == 0)[None]
    s = b.sum()
    if s > 0:
        b /= s
    return b.astype(dtype)


def map_like(H: int, W: int, seed: int, zero_frac: float = 0.3) -> np.ndarray:
    """A float32 [H][W] non-negative belief-map-like field (a fraction of exact zeros)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    m = rng.random((H, W)) ** 3
    m[rng.random((H, W)) < zero_frac] = 0.0
    return m.astype(np.float32)
