"""Algorithm 1's propagation in plain C (oracle, FP64): the same direct sums as
``oracle.filter.propagate``, in the same order, so the results are bit-identical (pinned by
``tests/test_oracle_filter.py``), with the channels spread over OpenMP threads.

TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT (see the package docstring).  It exists so that
the oracle can follow long trajectories on large grids (1000 steps of 256 x 256 x 72 states)
and so that the CPU baseline can be timed on one core and on all of them.

* ``propagate(B, M, corr, shifts, g, threads)``  Eq. 3 (AF, bilinear), Algorithm 1's mask,
  the 3-D blur of Eq. 7 as the direct triple sum, the mask and the edge correction of Eq. 8;
  no normalisation.
* ``Filter``  ``oracle.filter.Filter`` whose propagation runs here.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

from . import filter as F

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "prop.c")
_LIB = os.path.join(_HERE, "libprop.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile prop.c: FP64 with contraction off, no fast-math; OpenMP where the compiler has
    it (without it the threads argument is ignored)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-o", tmp, _SRC]
        try:
            subprocess.check_call(base + ["-fopenmp", "-lm"], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base + ["-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _c():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        lib.propagate_direct.restype = ctypes.c_int
        lib.propagate_direct.argtypes = [P, P, P, P, P] + [ctypes.c_int] * 6 + [P]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def propagate(B: np.ndarray, M: np.ndarray, corr: np.ndarray, shifts: np.ndarray, g: np.ndarray,
              threads: int = 1) -> np.ndarray:
    """``oracle.filter.propagate`` computed in C (bit-identical)."""
    K, H, W = B.shape
    B = np.ascontiguousarray(B, np.float64)
    M = np.ascontiguousarray(M, np.float64)
    corr = np.ascontiguousarray(np.broadcast_to(corr, B.shape), np.float64)
    shifts = np.ascontiguousarray(shifts, np.float64).reshape(K, 2)
    g = np.ascontiguousarray(g, np.float64)
    rk, r = g.shape[0] // 2, g.shape[1] // 2
    out = np.empty_like(B)
    if _c().propagate_direct(_ptr(B), _ptr(M), _ptr(corr), _ptr(shifts), _ptr(g), K, H, W, rk, r,
                             int(threads), _ptr(out)) != 0:
        raise MemoryError("propagate_direct: allocation failed")
    return out


def host_cores() -> int:
    """The cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


class Filter(F.Filter):
    """``oracle.filter.Filter`` with the propagation in C on `threads` threads."""

    def __init__(self, *args, threads: int = 1, **kw):
        super().__init__(*args, **kw)
        self.threads = threads

    def step(self, u: float, v: float, w: float) -> bool:
        self.odo.add(u, v, w)
        if not self.odo.due():
            return False
        T = propagate(self.B, self.M, self.corr, self.odo.shifts(), self.g, self.threads)
        self.odo.consume()
        self.B, Z, reinit = F.normalise(T, self.M)
        self.last_Z = Z
        if not reinit:
            self.logscale += math.log(Z)
        self.n_prop += 1
        return True
