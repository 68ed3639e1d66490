"""Anisotropic motion noise of Eq. 5-6 (oracle, FP64, direct sums).

Eq. 6 builds the covariance of the motion kernel from diag(sigma_x, sigma_y, sigma_theta)
rotated about z by the state's angle, and the text after Eq. 7 makes that angle the
channel's: G(B', k) is a 3-D convolution whose kernel depends on k.  With sigma_x ==
sigma_y the rotation drops out (``filter.motion_kernel``); here sigma_x != sigma_y.

Readings used (each also listed in the design notes):

* sigma_x acts along the heading of the output channel k, phi_k = 2 pi k / K + theta_t
  (theta_t after the message), and sigma_y across it: in the x/y plane
  Sigma_k = R(phi_k) diag(sigma_x^2, sigma_y^2) R(phi_k)^T, so an offset d = (di, dj)
  contributes d^T Sigma_k^-1 d = (d . e_k / sigma_x)^2 + (d . n_k / sigma_y)^2 with
  e_k = (cos phi_k, sin phi_k) and n_k = (-sin phi_k, cos phi_k).  (Eq. 6 writes
  R_z^T diag R_z; taking R_z as the map-to-robot rotation gives this form.)
* The theta part is independent (R_z leaves theta alone): the joint kernel of channel k is
  exp(-1/2 [d^T Sigma_k^-1 d + (dk / sigma_theta)^2]), sampled at integer offsets within
  radius r_xy (both x and y, ceil(3 max(sigma_x, sigma_y)) by default) and r_theta, and
  normalised to sum 1.
* T[k] = sum over (dk, dj, di) of g_k[dk][dj][di] * S[(k + dk) mod K][j + dj][i + di]: every
  source plane of output channel k is blurred with channel k's x/y kernel.
* G(B_0, k) of Alg. 1 / Eq. 8 is that convolution of the binary free tensor, so the edge
  correction has one plane per channel.
"""
from __future__ import annotations

import math

import numpy as np

from . import filter as F


def aniso_radius(sigma_x: float, sigma_y: float) -> int:
    """Truncation radius ceil(3 max(sigma_x, sigma_y)), the same in x and y."""
    return F.default_radius(max(sigma_x, sigma_y))


def rotated_kernel(phi: float, sigma_x: float, sigma_y: float, sigma_theta: float,
                   r_xy: int | None = None, r_theta: int | None = None) -> np.ndarray:
    """Eq. 5-6 for one output channel with heading phi: g[dk][dj][di], offsets -r..r,
    normalised so the whole kernel sums to 1."""
    r = aniso_radius(sigma_x, sigma_y) if r_xy is None else r_xy
    rt = F.default_radius(sigma_theta) if r_theta is None else r_theta
    dk = np.arange(-rt, rt + 1, dtype=np.float64)[:, None, None]
    dj = np.arange(-r, r + 1, dtype=np.float64)[None, :, None]
    di = np.arange(-r, r + 1, dtype=np.float64)[None, None, :]
    along = di * math.cos(phi) + dj * math.sin(phi)
    across = -di * math.sin(phi) + dj * math.cos(phi)
    q = (along / sigma_x) ** 2 + (across / sigma_y) ** 2
    if sigma_theta > 0:
        q = q + (dk / sigma_theta) ** 2
    else:
        q = q + np.where(dk == 0, 0.0, np.inf)
    g = np.exp(-0.5 * q)
    return g / g.sum()


def channel_kernels(K: int, theta_t: float, sigma_x: float, sigma_y: float, sigma_theta: float,
                    r_xy: int | None = None, r_theta: int | None = None) -> list:
    """The kernel of every output channel k (heading 2 pi k / K + theta_t)."""
    return [rotated_kernel(2.0 * math.pi * k / K + theta_t, sigma_x, sigma_y, sigma_theta, r_xy, r_theta)
            for k in range(K)]


def blur_per_channel(S: np.ndarray, kernels: list) -> np.ndarray:
    """G(S, k) for every k: the plain triple sum with channel k's kernel."""
    K = S.shape[0]
    T = np.zeros_like(S)
    for k in range(K):
        g = kernels[k]
        rk, r = g.shape[0] // 2, g.shape[1] // 2
        for a in range(-rk, rk + 1):
            Sk = S[(k + a) % K]
            for b in range(-r, r + 1):
                for c in range(-r, r + 1):
                    T[k] += g[a + rk, b + r, c + r] * F.take(Sk, b, c)
    return T


def edge_correction(M: np.ndarray, kernels: list) -> np.ndarray:
    """Eq. 8 per channel: 1 / G(B_0, k) on free cells, 0 on occupied ones; shape [K][H][W]."""
    K = len(kernels)
    G = blur_per_channel(np.broadcast_to(M, (K,) + M.shape).copy(), kernels)
    out = np.zeros_like(G)
    free = np.broadcast_to(M > 0, G.shape)
    out[free] = 1.0 / G[free]
    return out


def propagate(B: np.ndarray, M: np.ndarray, shifts: np.ndarray, kernels: list) -> np.ndarray:
    """Algorithm 1's propagation with the per-channel kernels (no normalisation)."""
    K = B.shape[0]
    S = np.stack([F.shift_bilinear(B[k], shifts[k, 0], shifts[k, 1]) for k in range(K)])
    S = M[None] * S
    T = M[None] * blur_per_channel(S, kernels)
    return T * edge_correction(M, kernels)


class Filter(F.Filter):
    """The session of ``filter.Filter`` with sigma_x (along the heading) != sigma_y."""

    def __init__(self, occ: np.ndarray, K: int, cell: float, sigma_x: float, sigma_y: float,
                 sigma_theta: float = 1.0, r_xy: int | None = None, r_theta: int | None = None,
                 min_shift_cells: float = 0.0):
        super().__init__(occ, K, cell, sigma_x, sigma_theta, r_xy, r_theta, min_shift_cells)
        self.sigma = (sigma_x, sigma_y, sigma_theta)
        self.radii = (r_xy, r_theta)

    def kernels(self) -> list:
        return channel_kernels(self.K, self.odo.theta, *self.sigma, *self.radii)

    def step(self, u: float, v: float, w: float) -> bool:
        self.odo.add(u, v, w)
        if not self.odo.due():
            return False
        T = propagate(self.B, self.M, self.odo.shifts(), self.kernels())
        self.odo.consume()
        self.B, Z, reinit = F.normalise(T, self.M)
        self.last_Z = Z
        if not reinit:
            self.logscale += math.log(Z)
        self.n_prop += 1
        return True
