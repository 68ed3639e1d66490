"""Pins of the FP64 oracle for Algorithm 1 (odometry shift, mask, 3-D blur, edge
normalisation, normaliser) against things other than itself: a library convolution, the
area-overlap geometry of Eq. 1's cell-uniform density, closed-form moments, invariants,
SE(2) composition, and the explicit transition matrix of Eq. 4 assembled from Kronecker
products on tiny grids."""
import math

import numpy as np
import pytest
from scipy import signal

from oracle import filter as F
from oracle import readout as R
from oracle.odometry import Odometry
from synth import fields, floorplan


def gauss1d(sigma, r):
    d = np.arange(-r, r + 1, dtype=np.float64)
    g = np.exp(-d * d / (2 * sigma * sigma)) if sigma > 0 else (d == 0).astype(float)
    return g / g.sum()


# ---------------------------------------------------------------- kernel (Eq. 5-6)

def test_kernel_closed_form_centre_and_ratios():
    g = F.motion_kernel(0.5, 1.0)
    assert g.shape == (7, 5, 5)
    assert abs(g.sum() - 1.0) < 1e-15
    zx = 1 + 2 * math.exp(-2) + 2 * math.exp(-8)
    zt = 1 + 2 * math.exp(-0.5) + 2 * math.exp(-2) + 2 * math.exp(-4.5)
    assert abs(g[3, 2, 2] - 1.0 / (zx * zx * zt)) < 1e-15
    assert abs(g[3, 2, 3] / g[3, 2, 2] - math.exp(-2)) < 1e-13
    assert abs(g[4, 2, 2] / g[3, 2, 2] - math.exp(-0.5)) < 1e-13
    assert abs(g[3, 0, 0] / g[3, 2, 2] - math.exp(-16)) < 1e-13


def test_kernel_is_product_of_1d_gaussians():
    g = F.motion_kernel(0.7, 1.3, 3, 4)
    prod = np.einsum("a,b,c->abc", gauss1d(1.3, 4), gauss1d(0.7, 3), gauss1d(0.7, 3))
    assert np.abs(g - prod).max() < 1e-15


def test_kernel_zero_sigma_is_delta():
    g = F.motion_kernel(0.0, 0.0)
    assert g.shape == (1, 1, 1) and g[0, 0, 0] == 1.0


# ---------------------------------------------------------------- AF shift (Eq. 3)

def overlap_shift(B, sx, sy):
    """Area-overlap transfer: source cell (j', i') translated by (sx, sy) overlaps output cell
    (j, i) in the product of the two 1-D interval overlaps (Eq. 1: uniform inside a cell)."""
    H, W = B.shape
    out = np.zeros_like(B)
    ov = lambda a, b: max(0.0, min(a + 1, b + 1) - max(a, b))
    for j in range(H):
        for i in range(W):
            acc = 0.0
            for jj in range(H):
                oy = ov(jj + sy, j)
                if oy == 0.0:
                    continue
                for ii in range(W):
                    ox = ov(ii + sx, i)
                    if ox:
                        acc += B[jj, ii] * ox * oy
            out[j, i] = acc
    return out


@pytest.mark.parametrize("sx,sy", [(0.3, -0.45), (-1.7, 2.25), (3.0, 0.5), (-0.01, 0.99)])
def test_shift_equals_area_overlap(sx, sy):
    rng = np.random.default_rng(1)
    B = rng.random((7, 9))
    assert np.abs(F.shift_bilinear(B, sx, sy) - overlap_shift(B, sx, sy)).max() < 1e-14


def test_integer_shift_is_exact_permutation():
    rng = np.random.default_rng(2)
    B = rng.random((6, 8))
    out = F.shift_bilinear(B, 2.0, -1.0)
    for j in range(6):
        for i in range(8):
            src_j, src_i = j + 1, i - 2
            want = B[src_j, src_i] if 0 <= src_j < 6 and 0 <= src_i < 8 else 0.0
            assert out[j, i] == want


def test_shift_conserves_interior_mass():
    B = np.zeros((20, 20))
    B[8:12, 7:13] = np.random.default_rng(3).random((4, 6))
    assert abs(F.shift_bilinear(B, 1.37, -2.61).sum() - B.sum()) < 1e-14


# ---------------------------------------------------------------- 3-D blur (Eq. 7)

def test_blur_matches_library_convolution():
    rng = np.random.default_rng(4)
    S = rng.random((6, 9, 11))
    g = F.motion_kernel(0.6, 0.9, 2, 2)
    padded = np.pad(S, ((2, 2), (0, 0), (0, 0)), mode="wrap")
    padded = np.pad(padded, ((0, 0), (2, 2), (2, 2)), mode="constant")
    want = signal.convolve(padded, g, mode="valid", method="direct")
    assert np.abs(F.blur3d(S, g) - want).max() < 1e-14


def test_blur_impulse_response_is_kernel():
    S = np.zeros((16, 15, 15))
    S[5, 7, 7] = 1.0
    g = F.motion_kernel(0.5, 1.0)
    T = F.blur3d(S, g)
    assert np.abs(T[2:9, 5:10, 5:10] - g).max() < 1e-16
    assert abs(T.sum() - 1.0) < 1e-15


# ---------------------------------------------------------------- edge normalisation (Eq. 8)

def test_edge_correction_straight_wall_closed_form():
    occ = np.zeros((21, 21), np.uint8)
    occ[:, 10] = 1                                   # one wall column, free elsewhere
    M = F.traversability(occ)
    g = F.motion_kernel(0.5, 1.0)
    corr = F.edge_correction(M, 4, g)
    gx = gauss1d(0.5, 2)
    # cell next to the wall (column 11), far from the border: the x-taps at -1 hit the wall
    assert abs(1.0 / corr[0, 10, 11] - (1.0 - gx[1])) < 1e-15
    assert abs(1.0 / corr[0, 10, 12] - (1.0 - gx[0])) < 1e-15   # tap -2 hits the wall
    assert abs(corr[0, 10, 15] - 1.0) < 1e-15
    assert (corr[:, :, 10] == 0).all()


def test_uniform_belief_stays_uniform_at_walls():
    """'Cliff vs wall' (Algorithm 1's edge correction): with zero motion a uniform belief is a fixed point."""
    occ = floorplan.rooms_map(5, size=32)
    flt = F.Filter(occ, 8, 0.1, 0.5, 1.0)
    B0 = flt.B.copy()
    flt.step(0.0, 0.0, 0.0)
    assert np.abs(flt.B - B0).max() < 1e-17
    assert abs(flt.last_Z - 1.0) < 1e-13


# ---------------------------------------------------------------- whole step invariants

def free_map(n):
    return np.zeros((n, n), np.uint8)


def test_a_mass_conserved_on_free_map():
    flt = F.Filter(free_map(48), 8, 0.1, 0.5, 1.0)
    flt.B[:] = 0
    rng = np.random.default_rng(5)
    flt.B[:, 16:32, 16:32] = rng.random((8, 16, 16))
    flt.B /= flt.B.sum()
    flt.step(0.23, -0.17, 0.05)                       # 2.3 cells and 1.7 cells
    assert abs(flt.last_Z - 1.0) < 1e-12


def test_b_zero_noise_integer_shift_is_permutation():
    """sigma = 0 (delta kernel) and an integer shift: the step is an exact permutation."""
    flt = F.Filter(free_map(24), 1, 1.0, 0.0, 0.0)
    rng = np.random.default_rng(6)
    B = np.zeros((1, 24, 24))
    B[:, 8:16, 8:16] = rng.random((1, 8, 8))
    B /= B.sum()
    flt.B = B.copy()
    flt.step(2.0, -3.0, 0.0)
    want = np.roll(np.roll(B, 2, 2), -3, 1)
    assert flt.last_Z == 1.0 or abs(flt.last_Z - 1.0) < 4e-16
    assert np.array_equal(flt.B * flt.last_Z, want)


def test_b_rotated_channels_shift_by_rotated_translation():
    """Channel k (heading k * 90 deg) moves by R(k * 90 deg) [2, 0]; cos(pi/2) is not exactly 0
    in FP64, so the match is to rounding."""
    flt = F.Filter(free_map(24), 4, 1.0, 0.0, 0.0)
    rng = np.random.default_rng(6)
    B = np.zeros((4, 24, 24))
    B[:, 8:16, 8:16] = rng.random((4, 8, 8))
    B /= B.sum()
    flt.B = B.copy()
    flt.step(2.0, 0.0, 0.0)
    want = np.stack([np.roll(B[0], 2, 1), np.roll(B[1], 2, 0),
                     np.roll(B[2], -2, 1), np.roll(B[3], -2, 0)])
    assert np.abs(flt.B - want).max() < 1e-15 * B.max()


def test_c_closed_form_moments_on_free_map():
    K, n = 1, 6
    flt = F.Filter(free_map(64), K, 1.0, 0.5, 1.0)
    flt.B[:] = 0
    flt.B[0, 20, 24] = 1.0
    s = np.array([0.3, 0.65])                         # cells per step; fractions 0.3 / 0.65
    for _ in range(n):
        flt.step(s[0], s[1], 0.0)
    b = flt.B[0]
    J, I = np.mgrid[0:64, 0:64]
    mx, my = (b * I).sum(), (b * J).sum()
    assert abs(mx - (24 + n * s[0])) < 1e-11
    assert abs(my - (20 + n * s[1])) < 1e-11
    gx = gauss1d(0.5, 2)
    var_g = (gx * np.arange(-2, 3) ** 2).sum()
    fx, fy = 1 - s[0], 1 - s[1]      # pull fractions: frac(-s) (the variance is symmetric in f)
    assert abs(((I - mx) ** 2 * b).sum() - n * (var_g + fx * (1 - fx))) < 1e-10
    assert abs(((J - my) ** 2 * b).sum() - n * (var_g + fy * (1 - fy))) < 1e-10


def test_c_theta_variance_grows_by_kernel_variance():
    K, n = 64, 4
    flt = F.Filter(free_map(12), K, 1.0, 0.0, 1.0)
    flt.B[:] = 0
    flt.B[30, 6, 6] = 1.0
    for _ in range(n):
        flt.step(0.0, 0.0, 0.0)
    prof = flt.B[:, 6, 6]
    k = np.arange(K)
    mean = (prof * k).sum()
    gt = gauss1d(1.0, 3)
    assert abs(mean - 30) < 1e-12
    assert abs(((k - 30) ** 2 * prof).sum() - n * (gt * np.arange(-3, 4) ** 2).sum()) < 1e-11


def test_d_occupied_cells_hold_no_mass():
    occ = floorplan.rooms_map(0)
    flt = F.Filter(occ, 16, 0.1)
    rng = np.random.default_rng(7)
    for _ in range(3):
        u, v, w = rng.normal(0, 0.07, 3)
        flt.step(u, v, w)
        assert (flt.B[:, occ != 0] == 0.0).all()
    assert abs(flt.B.sum() - 1.0) < 1e-12


def transition_matrix(occ, K, shifts, sigma_xy, sigma_th):
    """Eq. 4 as an explicit matrix on a tiny grid: T = diag(corr) diag(M) G diag(M) Shift, with
    Shift from the area overlap of translated cells and G = Gtheta (x) Gy (x) Gx built from 1-D
    Gaussians (circulant in theta, zero outside the grid in x/y)."""
    H, W = occ.shape
    M = (occ == 0).astype(float).reshape(-1)
    ov = lambda a, b: max(0.0, min(a + 1, b + 1) - max(a, b))
    n = H * W
    Sh = np.zeros((K * n, K * n))
    for k in range(K):
        sx, sy = shifts[k]
        for j in range(H):
            for i in range(W):
                for jj in range(H):
                    for ii in range(W):
                        w = ov(ii + sx, i) * ov(jj + sy, j)
                        if w:
                            Sh[k * n + j * W + i, k * n + jj * W + ii] = w
    rx = F.default_radius(sigma_xy)
    rt = F.default_radius(sigma_th)
    gx, gt = gauss1d(sigma_xy, rx), gauss1d(sigma_th, rt)
    Gx = np.zeros((W, W)); Gy = np.zeros((H, H)); Gt = np.zeros((K, K))
    for a in range(W):
        for b in range(W):
            if abs(a - b) <= rx:
                Gx[a, b] = gx[b - a + rx]
    for a in range(H):
        for b in range(H):
            if abs(a - b) <= rx:
                Gy[a, b] = gx[b - a + rx]
    for a in range(K):
        for d in range(-rt, rt + 1):
            Gt[a, (a + d) % K] += gt[d + rt]
    G = np.kron(Gt, np.kron(Gy, Gx))
    Mf = np.tile(M, K)
    GM = G @ Mf
    corr = np.where(Mf > 0, 1.0 / np.where(GM > 0, GM, 1.0), 0.0)
    return np.diag(corr) @ np.diag(Mf) @ G @ np.diag(Mf) @ Sh


@pytest.mark.parametrize("seed", [0, 1])
def test_e_brute_force_transition_matrix(seed):
    rng = np.random.default_rng(seed)
    H, W, K = 5, 6, 4
    occ = (rng.random((H, W)) < 0.25).astype(np.uint8)
    occ[2, 3] = 0
    flt = F.Filter(occ, K, 0.5, 0.7, 0.8)
    flt.B = F.uniform_belief(flt.M, K) * rng.random((K, H, W)) * 4
    flt.B /= flt.B.sum()
    b0 = flt.B.reshape(-1).copy()
    u, v, w = 0.31, -0.12, 0.2
    odo = Odometry(K, 0.5)
    odo.add(u, v, w)
    T = transition_matrix(occ, K, odo.shifts(), 0.7, 0.8)
    flt.step(u, v, w)
    nb = T @ b0
    assert np.abs(flt.B.reshape(-1) - nb / nb.sum()).max() < 1e-15
    assert abs(flt.last_Z - nb.sum()) < 1e-14
    # the pointwise evaluator agrees with the same matrix
    idx = [(k, j, i) for k in range(K) for j in range(H) for i in range(W)]
    pt = F.propagate_at(b0.reshape(K, H, W), flt.M, odo.shifts(), flt.g, idx)
    assert np.abs(pt - nb).max() < 1e-15


def test_all_mass_removed_restarts_uniform():
    occ = np.ones((6, 6), np.uint8)
    occ[2:4, 2:4] = 0
    flt = F.Filter(occ, 2, 1.0, 0.0, 0.0)
    flt.step(3.0, 0.0, 0.0)                           # everything moves onto walls
    assert flt.last_Z == 0.0
    assert np.abs(flt.B - F.uniform_belief(flt.M, 2)).max() == 0.0


# ---------------------------------------------------------------- odometry (Eq. 2, Alg. 1 gate)

def se2(x, y, t):
    return np.array([[math.cos(t), -math.sin(t), x], [math.sin(t), math.cos(t), y], [0, 0, 1]])


def test_channel0_gets_raw_translation_at_theta0():
    o = Odometry(8, 0.1)
    o.add(0.3, -0.2, 0.0)
    s = o.shifts()
    assert np.abs(s[0] - [3.0, -2.0]).max() < 1e-12
    assert np.abs(s[2] - [2.0, 3.0]).max() < 1e-12        # heading 90 deg


def test_accumulated_translation_matches_se2_composition():
    rng = np.random.default_rng(8)
    o = Odometry(16, 0.05)
    T = np.eye(3)
    for _ in range(12):
        u, v, w = rng.normal(0, 0.1, 3)
        o.add(u, v, w)
        T = T @ se2(u, v, w)
    assert np.abs(o.p - T[:2, 2]).max() < 1e-14
    assert abs(math.atan2(T[1, 0], T[0, 0]) - math.atan2(math.sin(o.theta), math.cos(o.theta))) < 1e-13


def test_gate_defers_small_motion():
    o = Odometry(4, 0.1, min_shift_cells=1.0)
    o.add(0.05, 0.0, 0.1)
    assert not o.due()
    o.add(0.06, 0.0, 0.0)
    assert o.due()


def test_estimate_of_a_point_mass_and_of_two_blobs():
    """The pose estimate's concentration and second hypothesis on beliefs with known answers:
    a point mass (all mass near, no second hypothesis); two blobs far apart (the near mass is
    the first blob's, the second hypothesis the other blob's peak); the disk's edge (a cell
    exactly radius_m away counts as near); the bin window wrapping around."""
    K, H, W, c = 8, 30, 40, 0.1
    b = np.zeros((K, H, W))
    b[3, 10, 12] = 1.0
    e = R.estimate(b, c, 0.25, 0.5, 1)
    assert (e["k"], e["j"], e["i"]) == (3, 10, 12) and e["mass_near"] == 1.0
    assert (e["second_j"], e["second_i"], e["second_p"]) == (-1, -1, 0.0)
    assert abs(e["x"] - 1.25) < 1e-12 and abs(e["y"] - 1.05) < 1e-12
    assert abs(e["theta"] - (2 * np.pi * 3 / 8 + 0.25)) < 1e-12
    # two blobs: 0.6 at bins 0 and 7 (wrapping) around (5, 5), 0.4 spread at (20, 30)
    b = np.zeros((K, H, W))
    b[0, 5, 5], b[7, 5, 6], b[1, 4, 5] = 0.3, 0.2, 0.1
    b[2, 20, 30], b[2, 21, 30] = 0.25, 0.15
    e = R.estimate(b, c, 0.0, 0.3, 1)
    assert (e["k"], e["j"], e["i"]) == (0, 5, 5)
    assert abs(e["mass_near"] - 0.6) < 1e-15                   # bin 7 is one bin from bin 0
    assert (e["second_j"], e["second_i"]) == (20, 30) and e["second_p"] == 0.25
    assert abs(e["second_ratio"] - 0.25 / 0.3) < 1e-15
    # the disk's edge: (5, 8) is exactly 0.3 m from (5, 5); (5, 9) is not
    b[0, 5, 8] = 0.01
    b[0, 5, 9] = 0.29
    e = R.estimate(b, c, 0.0, 0.3, 0)
    assert abs(e["mass_near"] - (0.3 + 0.1 * 0 + 0.01)) < 1e-15   # bins 7 and 1 are excluded
    assert (e["second_j"], e["second_i"]) == (5, 9)


# ------------------------------------------------------------------ the C restatement

@pytest.mark.parametrize("H,W,K,sxy,sth,shift", [
    (23, 31, 8, 0.5, 1.0, (0.37, -1.61)),      # ragged grid, sub-cell shift
    (16, 16, 3, 0.5, 1.2, (2.0, 0.0)),         # K below the theta ring (radius 4), integer shift
    (12, 40, 5, 0.0, 1.0, (-0.5, 0.25)),       # no x/y blur (radius 0)
    (9, 7, 4, 1.3, 0.0, (5.2, -7.9)),          # x/y radius 4 on a grid smaller than the window; no theta blur
])
def test_c_propagation_is_bit_identical_to_the_numpy_definition(H, W, K, sxy, sth, shift):
    """oracle.cprop restates Algorithm 1's propagation in C with the same double operations in
    the same order: every value equals the numpy definition's bit for bit, on any thread
    count (the threads split the channels, not the sums)."""
    from oracle import cprop
    rng = np.random.default_rng(H * W + K)
    occ = (rng.random((H, W)) < 0.2).astype(np.uint8)
    occ[0, 0] = 0
    M = F.traversability(occ)
    g = F.motion_kernel(sxy, sth)
    corr = F.edge_correction(M, K, g)
    B = fields.belief_like(occ, K, seed=H)
    sh = np.array([[shift[0] * math.cos(0.7 * k) - shift[1] * math.sin(0.7 * k),
                    shift[0] * math.sin(0.7 * k) + shift[1] * math.cos(0.7 * k)] for k in range(K)])
    want = F.propagate(B, M, corr, sh, g)
    for threads in (1, 3):
        got = cprop.propagate(B, M, corr, sh, g, threads)
        assert np.array_equal(got, want)


def test_c_filter_follows_the_numpy_filter():
    """The Filter on the C propagation follows the numpy Filter's trajectory bit for bit (the
    normalisation is the same numpy code)."""
    from oracle import cprop
    occ = floorplan.rooms_map(0, size=32)
    a = F.Filter(occ, 8, 0.1)
    b = cprop.Filter(occ, 8, 0.1, threads=2)
    rng = np.random.default_rng(0)
    for _ in range(5):
        u, v, w = rng.normal(0, 0.07, 3)
        a.step(u, v, w)
        b.step(u, v, w)
    assert np.array_equal(a.B, b.B) and a.logscale == b.logscale and a.last_Z == b.last_Z
