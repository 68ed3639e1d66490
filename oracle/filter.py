"""Belief-tensor update of Algorithm 1 (oracle, FP64, direct sums).

Layout: B[k][j][i] (channel k, row j = +y, column i = +x); M[j][i] = 1 on free cells and 0
on occupied ones (Section III-A.3 uses M this way: multiplying by it zeroes obstacles).

Readings of points the paper leaves open (each also listed in the design notes):

* AF (Eq. 3) with a sub-cell translation is the bilinear pull B'(i, j) = B(i - sx, j - sy),
  reading zero outside the grid.  Under the cell-uniform density of Eq. 1 this is exactly
  the area-overlap transfer of each cell's mass.
* Eq. 6's diag(sigma_x, sigma_y, sigma_theta) holds standard deviations, so the kernel of
  Eq. 5 is exp(-1/2 [(di/sx)^2 + (dj/sy)^2 + (dk/sth)^2]), sampled at integer offsets,
  truncated at radius ceil(3 sigma) per axis unless given, and normalised to sum 1.  With
  sigma_x == sigma_y the rotation R_z of Eq. 6 leaves it unchanged.
* The 3-D convolution of Eq. 7 is circular in theta and reads zero outside the grid in x/y.
* G(B_0, k) of Algorithm 1's edge correction (Eq. 8) is the same convolution applied to the binary tensor
  with ones on free cells; its pixel-wise inverse is taken on free cells only (occupied
  cells are zero after the mask that follows the blur anyway).
* The normaliser eta of Eq. 9 is applied after every propagation: Z = sum B, B /= Z.  If
  Z == 0 (all mass removed) the belief restarts uniform over free cells.
"""
from __future__ import annotations

import math

import numpy as np


def traversability(occ: np.ndarray) -> np.ndarray:
    """M of Section III-A.3: 1.0 on free cells, 0.0 on occupied ones."""
    return (np.asarray(occ) == 0).astype(np.float64)


def default_radius(sigma: float) -> int:
    """Truncation radius ceil(3 sigma); 0 for a zero sigma (a delta kernel)."""
    return 0 if sigma <= 0 else int(math.ceil(3.0 * sigma))


def motion_kernel(sigma_xy: float, sigma_theta: float, r_xy: int | None = None,
                  r_theta: int | None = None) -> np.ndarray:
    """Eq. 5 with the isotropic covariance of Eq. 6, as a joint 3-D array g[dk][dj][di]
    (offsets -r..r), normalised so the whole kernel sums to 1."""
    r_xy = default_radius(sigma_xy) if r_xy is None else r_xy
    r_th = default_radius(sigma_theta) if r_theta is None else r_theta
    dk = np.arange(-r_th, r_th + 1, dtype=np.float64)[:, None, None]
    dj = np.arange(-r_xy, r_xy + 1, dtype=np.float64)[None, :, None]
    di = np.arange(-r_xy, r_xy + 1, dtype=np.float64)[None, None, :]
    q = np.zeros((2 * r_th + 1, 2 * r_xy + 1, 2 * r_xy + 1))
    if sigma_xy > 0:
        q = q + (di / sigma_xy) ** 2 + (dj / sigma_xy) ** 2
    if sigma_theta > 0:
        q = q + (dk / sigma_theta) ** 2
    g = np.exp(-0.5 * q)
    return g / g.sum()


def take(A: np.ndarray, dj: int, di: int) -> np.ndarray:
    """out[..., j, i] = A[..., j + dj, i + di], zero where that index is off the grid."""
    H, W = A.shape[-2:]
    out = np.zeros_like(A)
    js, je = max(0, -dj), min(H, H - dj)
    is_, ie = max(0, -di), min(W, W - di)
    if js < je and is_ < ie:
        out[..., js:je, is_:ie] = A[..., js + dj:je + dj, is_ + di:ie + di]
    return out


def shift_bilinear(Bk: np.ndarray, sx: float, sy: float) -> np.ndarray:
    """Eq. 3 (AF, translation by (sx, sy) cells) with bilinear interpolation:
    out[j][i] = sum over the 4 neighbours of (i - sx, j - sy) of weight * Bk, zero off-grid."""
    x0, y0 = math.floor(-sx), math.floor(-sy)          # integer part of the source offset
    fx, fy = -sx - x0, -sy - y0                         # fractional part in [0, 1)
    return ((1 - fx) * (1 - fy) * take(Bk, y0, x0) + fx * (1 - fy) * take(Bk, y0, x0 + 1)
            + (1 - fx) * fy * take(Bk, y0 + 1, x0) + fx * fy * take(Bk, y0 + 1, x0 + 1))


def blur3d(S: np.ndarray, g: np.ndarray) -> np.ndarray:
    """Eq. 7: T[k][j][i] = sum_{dk,dj,di} g[dk][dj][di] * S[(k+dk) mod K][j+dj][i+di]."""
    rk, r = g.shape[0] // 2, g.shape[1] // 2
    T = np.zeros_like(S)
    for a in range(-rk, rk + 1):
        Sk = np.roll(S, -a, axis=0)                     # Sk[k] = S[(k + a) mod K]
        for b in range(-r, r + 1):
            for c in range(-r, r + 1):
                T += g[a + rk, b + r, c + r] * take(Sk, b, c)
    return T


def edge_correction(M: np.ndarray, K: int, g: np.ndarray) -> np.ndarray:
    """Algorithm 1's edge correction (Eq. 8): the pixel-wise inverse of G(B_0, k), where B_0 is the binary
    tensor with ones on free cells; zero on occupied cells.  Shape [K][H][W]."""
    G = blur3d(np.broadcast_to(M, (K,) + M.shape).copy(), g)
    out = np.zeros_like(G)
    free = np.broadcast_to(M > 0, G.shape)
    out[free] = 1.0 / G[free]
    return out


def uniform_belief(M: np.ndarray, K: int) -> np.ndarray:
    """All free states equally likely (Section III-A: the initial state is unknown)."""
    n = M.sum()
    return np.broadcast_to(M / (K * n), (K,) + M.shape).copy()


def propagate(B: np.ndarray, M: np.ndarray, corr: np.ndarray, shifts: np.ndarray,
              g: np.ndarray) -> np.ndarray:
    """Algorithm 1's propagation for every channel k (no normalisation):
    B' = AF(B, u_k); B' = M * B'; B'' = G(B'); B'' = M * B''; B_t = B'' * G(B_0)^-1."""
    K = B.shape[0]
    S = np.stack([shift_bilinear(B[k], shifts[k, 0], shifts[k, 1]) for k in range(K)])
    S = M[None] * S
    T = blur3d(S, g)
    T = M[None] * T
    return T * corr


def propagate_at(B: np.ndarray, M: np.ndarray, shifts: np.ndarray, g: np.ndarray,
                 idx) -> np.ndarray:
    """Algorithm 1's propagation (no normalisation) evaluated at the requested states only, each one
    from the definitions: for output (k, j, i) on a free cell,
        T = sum_{dk,dj,di} g[dk][dj][di] * M(j+dj, i+di) * AF(B, s)[(k+dk) mod K](j+dj, i+di)
        G = sum_{dk,dj,di} g[dk][dj][di] * M(j+dj, i+di)           (G(B_0, k), Eq. 8)
    and the result is T / G (0 on occupied cells).  AF is the bilinear pull of Eq. 3."""
    K, H, W = B.shape
    rk, r = g.shape[0] // 2, g.shape[1] // 2

    def af(kk, jj, ii):
        sx, sy = shifts[kk]
        x, y = ii - sx, jj - sy
        x0, y0 = math.floor(x), math.floor(y)
        fx, fy = x - x0, y - y0
        v = 0.0
        for (dy, wy) in ((0, 1 - fy), (1, fy)):
            for (dx, wx) in ((0, 1 - fx), (1, fx)):
                yy, xx = y0 + dy, x0 + dx
                if 0 <= yy < H and 0 <= xx < W:
                    v += wy * wx * B[kk, yy, xx]
        return v

    out = np.zeros(len(idx))
    for n, (k, j, i) in enumerate(idx):
        if M[j, i] == 0:
            continue
        T = G = 0.0
        for a in range(-rk, rk + 1):
            kk = (k + a) % K
            for b in range(-r, r + 1):
                jj = j + b
                if not 0 <= jj < H:
                    continue
                for c in range(-r, r + 1):
                    ii = i + c
                    if not 0 <= ii < W or M[jj, ii] == 0:
                        continue
                    w = g[a + rk, b + r, c + r]
                    G += w
                    T += w * af(kk, jj, ii)
        out[n] = T / G
    return out


def normalise(B: np.ndarray, M: np.ndarray):
    """Eq. 9's eta: divide by Z = sum B.  Returns (B / Z, Z, reinit); Z == 0 restarts from
    the uniform belief over free cells."""
    Z = float(B.sum())
    if not Z > 0.0:
        return uniform_belief(M, B.shape[0]), Z, True
    return B / Z, Z, False


class Filter:
    """The whole odometry + map update as the library's session API exposes it."""

    def __init__(self, occ: np.ndarray, K: int, cell: float, sigma_xy: float = 0.5,
                 sigma_theta: float = 1.0, r_xy: int | None = None, r_theta: int | None = None,
                 min_shift_cells: float = 0.0):
        from .odometry import Odometry
        self.M = traversability(occ)
        self.K = K
        self.g = motion_kernel(sigma_xy, sigma_theta, r_xy, r_theta)
        self.corr = edge_correction(self.M, K, self.g)
        self.B = uniform_belief(self.M, K)
        self.odo = Odometry(K, cell, min_shift_cells)
        self.logscale = 0.0
        self.last_Z = 1.0
        self.n_prop = 0

    def step(self, u: float, v: float, w: float) -> bool:
        """One odometry message; returns True when the belief was propagated."""
        self.odo.add(u, v, w)
        if not self.odo.due():
            return False
        T = propagate(self.B, self.M, self.corr, self.odo.shifts(), self.g)
        self.odo.consume()
        self.B, Z, reinit = normalise(T, self.M)
        self.last_Z = Z
        if not reinit:
            self.logscale += math.log(Z)
        self.n_prop += 1
        return True
