"""Per-element error bounds of the reduced-precision storage, shared by the GPU parity tests.

A BF16 store (error diffusion along theta) returns one of the two BF16 neighbours of its FP32
input, so its error is below one BF16 unit in the last place of that value: 2^(e - 7) for a
value in [2^e, 2^(e+1)) (8 significant bits).  Before the store, the FP32 arithmetic of one
propagation (about 30 rounded operations on non-negative terms) is within a few 1e-6 of the
value itself.  The bound of one stored BF16 result is therefore

    |stored - exact| <= ulp_bf16(exact * (1 + 1e-5)) + 5e-6 * exact

per element (the factor 1 + 1e-5 covers an FP32 value that crossed into the next binade).
"""
import numpy as np


def bf16_ulp(x) -> np.ndarray:
    """One BF16 unit in the last place of each (non-negative) value; 0 for 0."""
    x = np.asarray(x, np.float64)
    out = np.zeros_like(x)
    pos = x > 0
    out[pos] = np.exp2(np.floor(np.log2(x[pos])) - 7.0)
    return out


def bf16_step_bound(exact, fp32_rel: float = 5e-6) -> np.ndarray:
    """Per-element bound of one propagation stored in BF16 (see the module docstring)."""
    exact = np.asarray(exact, np.float64)
    return bf16_ulp(exact * (1.0 + 1e-5)) + fp32_rel * exact
