"""Dense scan update with a precomputed expected-range table (oracle, test infrastructure only).

Eq. 9 applied to every state instead of a dithered sample: the map is static, so the expected
range of every cell along a fixed set of directions can be cast once and stored; a scan then
scores every (cell, bin) state from that table and reweights the whole tensor, with eta the
global normaliser.

Readings used (each also listed in the design notes):

* The table holds A directions 2 pi a / A, a = 0 .. A-1, with A a multiple of K, so bin k's
  heading 2 pi k / K is table direction k A / K.  A direction's unit vector is computed in
  FP64 and rounded to FP32 (as for the sampled update's beams).
* Entry (a, j, i) is the FP32 grid walk ``dda_cells`` from the centre of cell (j, i) along
  direction a, capped at r_max (in cells: float32(r_max / cell)), quantised to 8 bits:
  q = floor(t * inv_step + 0.5), capped at 255, inv_step = float32(255 / rmax_cells), in
  FP32 with each operation rounded.  The range it stands for is q * float32(r_max / 255) m.
* Beam b of a state in bin k looks up direction (k A / K + m_b) mod A, where
  m_b = floor(x + 0.5) mod A and x = (theta_t + (angle_min + angle_inc b)) / (2 pi / A),
  evaluated in FP64 in that order: the beam's offset from the bin heading, rounded to the
  nearest table direction (an angular error of at most pi / A).
* log P(z | x) as in the sampled update: independent beams, every ``beam_stride``-th beam,
  beams with z_b >= r_max skipped, Gaussian in the range error with sigma_r.
* Eq. 9: b <- b w / sum(b w) over all states with w = exp(log L - max log L), the maximum
  taken over the states of free cells.  Occupied cells hold no mass and stay 0.
* The log-scale grows by the log of Eq. 9's normaliser: log(sum(b w)) + max log L (b the
  normalised belief before the update).
"""
from __future__ import annotations

import math

import numpy as np

from . import lidar


def table_dirs32(A: int) -> np.ndarray:
    """Unit vectors of the table directions 2 pi a / A: FP64 cos / sin rounded to FP32, (A, 2)."""
    d = np.empty((A, 2), np.float32)
    for a in range(A):
        ang = (2.0 * math.pi / A) * a
        d[a, 0] = np.float32(math.cos(ang))
        d[a, 1] = np.float32(math.sin(ang))
    return d


def quant(r_max: float, cell: float):
    """(rmax_cells, inv_step, step_m): the walk's cap in cells, the FP32 code scale and the
    range one code step stands for (metres)."""
    rmax_cells = np.float32(r_max / cell)
    inv_step = np.float32(255.0 / float(rmax_cells))
    step_m = np.float32(r_max / 255.0)
    return rmax_cells, inv_step, step_m


def range_table(occ: np.ndarray, A: int, r_max: float, cell: float) -> np.ndarray:
    """uint8 [A][H][W]: the quantised walk range from every cell along every table direction."""
    occ = np.ascontiguousarray(occ, dtype=np.uint8)
    H, W = occ.shape
    rmax_cells, inv_step, _ = quant(r_max, cell)
    dirs = np.ascontiguousarray(table_dirs32(A))
    out = np.empty((A, H, W), np.uint8)
    lidar._ref().range_table(lidar._ptr(occ), H, W, lidar._ptr(dirs), A,
                             lidar.ctypes.c_float(rmax_cells), lidar.ctypes.c_float(inv_step),
                             lidar._ptr(out))
    return out


def beam_offsets(theta: float, angle_min: float, angle_inc: float, z: np.ndarray, r_max: float,
                 beam_stride: int, A: int):
    """The used beams (b % stride == 0, z_b < r_max): their table offsets m_b and ranges."""
    m, zu = [], []
    for b in range(0, len(z), beam_stride):
        if not z[b] < r_max:
            continue
        x = (theta + (angle_min + angle_inc * b)) / (2.0 * math.pi / A)
        m.append(int(math.floor(x + 0.5)) % A)
        zu.append(float(z[b]))
    return np.array(m, np.int64), np.array(zu, np.float64)


def log_likelihood(table: np.ndarray, K: int, m: np.ndarray, zu: np.ndarray, r_max: float,
                   sigma_r: float) -> np.ndarray:
    """log P(z | x) of every state [K][H][W] from the table (FP64)."""
    A = table.shape[0]
    s = A // K
    step = float(np.float32(r_max / 255.0))
    out = np.zeros((K,) + table.shape[1:])
    for k in range(K):
        for mb, z in zip(m, zu):
            r = table[(k * s + mb) % A].astype(np.float64) * step
            d = z - r
            out[k] -= d * d
    return out / (2.0 * sigma_r * sigma_r)


def dense_update(b: np.ndarray, occ: np.ndarray, table: np.ndarray, theta: float, z: np.ndarray,
                 angle_min: float, angle_inc: float, r_max: float, beam_stride: int, sigma_r: float):
    """Eq. 9 on every state.  Returns (new belief, log L, max log L, log of the normaliser)."""
    K = b.shape[0]
    A = table.shape[0]
    if A % K:
        raise ValueError("the table's direction count must be a multiple of K")
    m, zu = beam_offsets(theta, angle_min, angle_inc, z, r_max, beam_stride, A)
    logL = log_likelihood(table, K, m, zu, r_max, sigma_r)
    free = np.broadcast_to(occ == 0, b.shape)
    mx = logL[free].max()
    w = np.where(free, np.exp(logL - mx), 0.0)
    bw = b * w
    S = bw.sum()
    return bw / S, logL, mx, math.log(S) + mx


class Filter:
    """A session of ``filter.Filter`` plus the dense scan update (wraps an existing filter)."""

    def __init__(self, f, occ: np.ndarray, cell: float, A: int, r_max: float):
        self.f = f
        self.occ = np.ascontiguousarray(occ, dtype=np.uint8)
        self.r_max = r_max
        self.table = range_table(self.occ, A, r_max, cell)

    def dense_update(self, z: np.ndarray, angle_min: float, angle_inc: float, beam_stride: int,
                     sigma_r: float):
        self.f.B, _, _, dl = dense_update(self.f.B, self.occ, self.table, self.f.odo.theta, z,
                                          angle_min, angle_inc, self.r_max, beam_stride, sigma_r)
        self.f.logscale += dl


def probe_scan(table: np.ndarray, K: int, cell_index: int, probe_bin: int, beam_step: int):
    """The noise-free scan of a probe: beams b = 0, 1, ... on table directions
    probe_bin A/K + b beam_step (mod A), b beam_step < A; each range is the table's code at the
    probe's cell (in code steps).  Returns the used beams' offsets m_b = b beam_step and codes
    (code 255, the capped range, is skipped like a dropout)."""
    A = table.shape[0]
    s = A // K
    col = table.reshape(A, -1)[:, cell_index]
    m, q = [], []
    for b in range(0, (A + beam_step - 1) // beam_step):
        off = b * beam_step
        if off >= A:
            break
        code = int(col[(probe_bin * s + off) % A])
        if code == 255:
            continue
        m.append(off)
        q.append(code)
    return np.array(m, np.int64), np.array(q, np.int64)


def map_difficulty(occ: np.ndarray, table: np.ndarray, K: int, cell: float, r_max: float,
                   probes: np.ndarray, probe_bin: int, beam_step: int, sigma_r: float, C: float):
    """Eq. 11 on a set of probe cells: for each probe p, the state that best matches its
    noise-free scan (the argmax of log L over the states of free cells, the first in [K][H][W]
    order on ties) gives the location p_hat; e_p = |p - p_hat| between cell centres (m).
    Returns (e_p for every probe, the number with e_p > C)."""
    H, W = occ.shape
    step = float(np.float32(r_max / 255.0))
    free = np.broadcast_to(occ == 0, (K, H, W))
    errors = []
    for p in probes:
        m, q = probe_scan(table, K, int(p), probe_bin, beam_step)
        logL = log_likelihood(table, K, m, q.astype(np.float64) * step, r_max, sigma_r)
        logL = np.where(free, logL, -np.inf)
        flat = int(np.argmax(logL.reshape(-1)))
        rem = flat % (H * W)
        jh, ih = divmod(rem, W)
        j, i = divmod(int(p), W)
        errors.append(cell * math.hypot(jh - j, ih - i))
    e = np.array(errors)
    return e, int((e > C).sum())
