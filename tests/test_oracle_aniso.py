"""Pins of the anisotropic motion kernel (Eq. 5-6, oracle ``aniso``) to facts other than its
own formula: the isotropic special case, the covariance and orientation of the kernel (its
second moments), equivariance under a 90-degree rotation of the world, mass conservation on a
free map, and the heading alignment of a blurred point mass."""
import math

import numpy as np
import pytest

from oracle import aniso as A
from oracle import filter as F


def test_isotropic_case_is_the_separable_kernel():
    for phi in (0.0, 0.3, 1.9, -2.5):
        g = A.rotated_kernel(phi, 0.5, 0.5, 1.0)
        assert np.allclose(g, F.motion_kernel(0.5, 1.0), rtol=0, atol=1e-15)


def test_isotropic_filter_reproduces_the_isotropic_trajectory():
    rng = np.random.default_rng(0)
    occ = (rng.random((14, 17)) < 0.15).astype(np.uint8)
    a = A.Filter(occ, 8, 0.1, 0.5, 0.5, 1.0)
    b = F.Filter(occ, 8, 0.1, 0.5, 1.0)
    for u, v, w in [(0.03, 0.01, 0.4), (-0.05, 0.02, -0.2), (0.0, 0.0, 1.1)]:
        a.step(u, v, w)
        b.step(u, v, w)
        assert np.abs(a.B - b.B).max() < 1e-13


@pytest.mark.parametrize("phi", [0.0, 0.4, math.pi / 2, 2.3])
def test_kernel_second_moments_are_the_rotated_covariance(phi):
    sx, sy = 1.6, 0.8
    g = A.rotated_kernel(phi, sx, sy, 0.0, r_xy=9)[0]
    r = g.shape[0] // 2
    J, I = np.mgrid[-r:r + 1, -r:r + 1].astype(np.float64)
    assert abs((g * I).sum()) < 1e-12 and abs((g * J).sum()) < 1e-12
    C = np.array([[(g * I * I).sum(), (g * I * J).sum()], [(g * I * J).sum(), (g * J * J).sum()]])
    R = np.array([[math.cos(phi), -math.sin(phi)], [math.sin(phi), math.cos(phi)]])
    want = R @ np.diag([sx * sx, sy * sy]) @ R.T
    assert np.abs(C - want).max() < 2e-3                     # sampling error of a lattice Gaussian
    w, V = np.linalg.eigh(C)                                  # the long axis points along phi
    axis = V[:, 1]
    assert abs(abs(axis @ np.array([math.cos(phi), math.sin(phi)])) - 1.0) < 1e-3


def test_rotating_the_world_by_90_degrees_commutes_with_a_step():
    """Rotating the map and the belief by +90 degrees and moving every hypothesis to the channel
    a quarter turn further commutes with a step (the same odometry, relative to the robot)."""
    K, n = 8, 13
    rng = np.random.default_rng(3)
    occ = (rng.random((n, n)) < 0.15).astype(np.uint8)
    B = rng.random((K, n, n)) * (occ == 0)
    B /= B.sum()

    def rot(A_):          # +90 degrees: (x, y) -> (-y, x) with row = +y, column = +x
        return np.flip(np.swapaxes(A_, -1, -2), axis=-1)

    f1 = A.Filter(occ, K, 0.1, 1.1, 0.5, 0.9)
    f1.B = B.copy()
    f2 = A.Filter(rot(occ), K, 0.1, 1.1, 0.5, 0.9)
    f2.B = np.roll(rot(B), K // 4, axis=0)
    for u, v, w in [(0.07, -0.03, 0.3), (0.02, 0.05, -0.6)]:
        f1.step(u, v, w)
        f2.step(u, v, w)
        assert np.abs(np.roll(rot(f1.B), K // 4, axis=0) - f2.B).max() < 1e-13


def test_mass_is_conserved_on_a_free_map():
    K, n = 8, 31
    occ = np.zeros((n, n), np.uint8)
    B = np.zeros((K, n, n))
    B[:, 12:19, 12:19] = np.random.default_rng(1).random((K, 7, 7))
    B /= B.sum()
    f = A.Filter(occ, K, 0.1, 1.2, 0.6, 1.0)
    f.B = B
    f.step(0.12, -0.07, 0.5)
    assert abs(f.last_Z - 1.0) < 1e-12


def test_a_point_mass_spreads_along_each_channels_heading():
    K, n = 8, 41
    occ = np.zeros((n, n), np.uint8)
    f = A.Filter(occ, K, 0.1, 1.5, 0.5, 0.0)           # no theta blur: channels stay apart
    f.B = np.zeros((K, n, n))
    f.B[:, n // 2, n // 2] = 1.0 / K
    theta = 0.35
    f.step(0.0, 0.0, theta)                              # heading offset only, zero shift
    J, I = np.mgrid[0:n, 0:n].astype(np.float64)
    for k in range(K):
        p = f.B[k] / f.B[k].sum()
        mi, mj = (p * I).sum(), (p * J).sum()
        C = np.array([[(p * (I - mi) ** 2).sum(), (p * (I - mi) * (J - mj)).sum()],
                      [(p * (I - mi) * (J - mj)).sum(), (p * (J - mj) ** 2).sum()]])
        axis = np.linalg.eigh(C)[1][:, 1]
        phi = 2 * math.pi * k / K + theta
        assert abs(abs(axis @ np.array([math.cos(phi), math.sin(phi)])) - 1.0) < 2e-3, k
