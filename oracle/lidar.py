"""LIDAR sample update of Section III-B (oracle).

Steps, in the paper's order:
1. belief map m = max over channels (Section III-A.3, end);
2. Floyd-Steinberg selection of sample cells that follow m (Section III-B.1, Fig. 1c) --
   ``fs_select`` in ``ref.c`` (FP32, fixed order);
3. for every sampled cell and every channel, the likelihood P(z | x) of Eq. 9 from the
   expected ranges of a grid ray cast (``dda_cells`` in ``ref.c``, FP32) -- FP64 scoring;
4. Eq. 9 on the sampled states: multiply by the likelihood and renormalise.

Readings of what the paper leaves open:
* FS input: v = min(1, N_s * m / sum(m)), so about N_s cells are selected; the FP32 factor
  fs = N_s / sum(m) is an input of ``fs_select``.
* Every channel of a sampled cell is a sampled state.
* P(z | x) (the paper's LIDAR model comes from its simulator and is not given): independent
  beams, Gaussian in the range error, sigma_r; only every ``beam_stride``-th beam is used,
  and beams that returned r_max (no return / dropout) are skipped.  Beam b of a state in
  channel k points at k*dTheta + theta_t + angle_min + b*angle_inc.
* Eq. 9's eta is applied within the sampled set: the set keeps its total mass, so
  unsampled states keep their value and the tensor still sums to 1.  Weights are
  proportional to L b over the set, normalised in the log domain.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ref.c")
_LIB = os.path.join(_HERE, "libref.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ref.c with the host C compiler: FP32 with contraction off, no fast-math."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                               "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _ref():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        lib.fs_select.restype = ctypes.c_int
        lib.fs_select.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_float, P]
        lib.dda_cells.restype = ctypes.c_float
        lib.dda_cells.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                  ctypes.c_float, ctypes.c_float, ctypes.c_float]
        lib.dda_ranges.restype = None
        lib.dda_ranges.argtypes = [P, ctypes.c_int, ctypes.c_int, P, ctypes.c_int, P,
                                   ctypes.c_int, ctypes.c_float, ctypes.c_float, P]
        lib.range_table.restype = None
        lib.range_table.argtypes = [P, ctypes.c_int, ctypes.c_int, P, ctypes.c_int,
                                    ctypes.c_float, ctypes.c_float, P]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def fs_factor(m: np.ndarray, n_samples: int) -> np.float32:
    """fs = N_s / sum(m) (FP64 sum), rounded to FP32."""
    return np.float32(n_samples / float(np.asarray(m, np.float64).sum()))


def fs_select(m32: np.ndarray, fs: float) -> np.ndarray:
    """Section III-B.1: uint8 [H][W] selection mask (FP32 Floyd-Steinberg)."""
    m32 = np.ascontiguousarray(m32, dtype=np.float32)
    H, W = m32.shape
    sel = np.zeros((H, W), np.uint8)
    n = _ref().fs_select(_ptr(m32), H, W, ctypes.c_float(fs), _ptr(sel))
    if n < 0:
        raise MemoryError("fs_select")
    return sel


def samples_from_mask(sel: np.ndarray) -> np.ndarray:
    """Sampled cells as linear indices j*W + i in raster order."""
    return np.flatnonzero(sel.reshape(-1)).astype(np.int32)


def beam_angles(K: int, theta: float, angle_min: float, angle_inc: float, n_beams: int,
                beam_stride: int) -> np.ndarray:
    """Map-frame angle (FP64) of every used beam b (b % stride == 0) of a state in channel k:
    k * (2 pi / K) + theta_t + (angle_min + angle_inc * b).  Shape (K, n_used)."""
    bs = list(range(0, n_beams, beam_stride))
    out = np.empty((K, len(bs)))
    for k in range(K):
        for n, b in enumerate(bs):
            out[k, n] = (2.0 * math.pi / K) * k + theta + (angle_min + angle_inc * b)
    return out


def beam_dirs32(angles: np.ndarray) -> np.ndarray:
    """Unit directions (cos, sin) of each angle, computed in FP64 by libm, rounded to FP32."""
    flat = angles.reshape(-1)
    d = np.empty((flat.size, 2), np.float32)
    for n, a in enumerate(flat):
        d[n, 0] = np.float32(math.cos(a))
        d[n, 1] = np.float32(math.sin(a))
    return d.reshape(angles.shape + (2,))


def dda_cells(occ: np.ndarray, j: int, i: int, dx: float, dy: float, rmax_cells: float) -> float:
    occ = np.ascontiguousarray(occ, dtype=np.uint8)
    H, W = occ.shape
    return float(_ref().dda_cells(_ptr(occ), H, W, j, i, ctypes.c_float(dx),
                                  ctypes.c_float(dy), ctypes.c_float(rmax_cells)))


def expected_ranges(occ: np.ndarray, cells: np.ndarray, dirs32: np.ndarray, r_max: float,
                    cell: float) -> np.ndarray:
    """FP32 expected range (m) for each sampled cell and each direction: shape
    (n_cells,) + dirs32.shape[:-1].  The cap is float32(r_max / cell) cells and the
    conversion to metres multiplies by float32(cell)."""
    occ = np.ascontiguousarray(occ, dtype=np.uint8)
    H, W = occ.shape
    cells = np.ascontiguousarray(cells, dtype=np.int32)
    d = np.ascontiguousarray(dirs32.reshape(-1, 2), dtype=np.float32)
    out = np.empty((cells.size, d.shape[0]), np.float32)
    _ref().dda_ranges(_ptr(occ), H, W, _ptr(cells), int(cells.size), _ptr(d), int(d.shape[0]),
                      ctypes.c_float(np.float32(r_max / cell)), ctypes.c_float(np.float32(cell)),
                      _ptr(out))
    return out.reshape((cells.size,) + dirs32.shape[:-1])


def log_likelihood(ranges: np.ndarray, z: np.ndarray, r_max: float, beam_stride: int,
                   sigma_r: float) -> np.ndarray:
    """log P(z | x) for each state: sum over used beams with z_b < r_max of
    -(z_b - r_hat)^2 / (2 sigma_r^2) (FP64).  ranges: (n_cells, K, n_used)."""
    zu = np.asarray(z, np.float64)[::beam_stride]
    use = zu < r_max
    d = zu[None, None, :] - ranges.astype(np.float64)
    return -(d * d * use[None, None, :]).sum(axis=2) / (2.0 * sigma_r * sigma_r)


def reweight(b: np.ndarray, cells: np.ndarray, logL: np.ndarray) -> np.ndarray:
    """Eq. 9 on the sampled states (all channels of each sampled cell), keeping the set's
    total mass A = sum_set b: b(c,k) <- A L(c,k) b(c,k) / sum_set L b.  The products L b are
    formed as exp(log L + log b - c) with c their largest logarithm, the same values as
    b exp(log L - max log L) * A / sum(b exp(log L - max log L)) but without underflow when the
    scan's likelihood peaks on states of tiny or zero belief.  States with b = 0 stay 0; a set
    without mass is left as it is."""
    K, H, W = b.shape
    out = b.copy()
    if cells.size == 0:
        return out
    flat = out.reshape(K, H * W)
    sub = flat[:, cells].T                          # (n_cells, K)
    mass = sub.sum()
    if not mass > 0.0:
        return out
    pos = sub > 0.0
    lw = np.full(sub.shape, -np.inf)
    lw[pos] = logL[pos] + np.log(sub[pos])
    w = np.where(pos, np.exp(lw - lw.max()), 0.0)
    flat[:, cells] = (w * (mass / w.sum())).T
    return out


def lidar_update(b: np.ndarray, occ: np.ndarray, theta: float, z: np.ndarray, cell: float,
                 angle_min: float, angle_inc: float, r_max: float, beam_stride: int,
                 sigma_r: float, n_samples: int, cells: np.ndarray | None = None):
    """The whole sample update.  `cells` overrides the FS selection (same list for two
    implementations); returns (new belief, sampled cells)."""
    K = b.shape[0]
    if cells is None:
        m = b.max(axis=0)
        m32 = m.astype(np.float32)
        cells = samples_from_mask(fs_select(m32, fs_factor(m32, n_samples)))
    ang = beam_angles(K, theta, angle_min, angle_inc, len(z), beam_stride)
    r = expected_ranges(occ, cells, beam_dirs32(ang), r_max, cell)
    logL = log_likelihood(r, z, r_max, beam_stride, sigma_r)
    return reweight(b, cells, logL), cells
