"""Pins of the oracle's LIDAR sample update (Section III-B): Floyd-Steinberg selection against
hand-worked and textbook results, the grid ray cast against analytic wall distances and a
brute-force fine ray march, and the Eq. 9 reweighting against its invariants and the
observation condition of Eq. 10."""
import math

import numpy as np
import pytest

from oracle import lidar as L
from synth import floorplan, scan


# ---------------------------------------------------------------- Floyd-Steinberg (III-B.1)

def test_fs_hand_worked_2x2():
    # v = 0.5 everywhere (m = 0.5, fs = 1).  By hand, with exact binary fractions:
    # (0,0): 0.5 >= 0.5 -> on,  err -0.5: right -0.21875, down -0.15625, down-right -0.03125
    # (0,1): 0.5 - 0.21875 = 0.28125 -> off; down-left +0.052734375, down +0.087890625
    # (1,0): 0.5 - 0.15625 + 0.052734375 = 0.396484375 -> off; right +0.173461914...
    # (1,1): 0.5 - 0.03125 + 0.087890625 + 0.1734619140625 = 0.7301025390625 -> on
    sel = L.fs_select(np.full((2, 2), 0.5, np.float32), 1.0)
    assert sel.tolist() == [[1, 0], [0, 1]]


def test_fs_half_grey_is_checkerboard():
    """The textbook Floyd-Steinberg result for 50 % grey: a checkerboard."""
    sel = L.fs_select(np.full((16, 16), 0.5, np.float32), 1.0)
    J, I = np.mgrid[0:16, 0:16]
    assert (sel == ((I + J) % 2 == 0)).all()


def test_fs_extremes_and_clamp():
    assert L.fs_select(np.zeros((5, 7), np.float32), 3.0).sum() == 0
    assert L.fs_select(np.full((5, 7), 2.0, np.float32), 1.0).sum() == 35    # clamped to 1
    one = np.zeros((9, 9), np.float32)
    one[4, 4] = 1.0
    sel = L.fs_select(one, 1.0)
    assert sel.sum() == 1 and sel[4, 4] == 1


@pytest.mark.parametrize("level", [0.25, 0.1, 0.8])
def test_fs_density_follows_grey_level(level):
    n = 64
    sel = L.fs_select(np.full((n, n), level, np.float32), 1.0)
    assert abs(sel.sum() - level * n * n) <= 2 * n


def test_fs_count_tracks_total_value():
    rng = np.random.default_rng(3)
    m = (rng.random((50, 70)) ** 3).astype(np.float32)
    fs = L.fs_factor(m, 400)
    sel = L.fs_select(m, float(fs))
    v = np.minimum(1.0, m.astype(np.float64) * float(fs))
    assert abs(int(sel.sum()) - v.sum()) <= 50 + 70


# ---------------------------------------------------------------- grid ray cast

def walled(n):
    occ = np.zeros((n, n), np.uint8)
    occ[0, :] = occ[-1, :] = occ[:, 0] = occ[:, -1] = 1
    return occ


@pytest.mark.parametrize("deg", [0.0, 7.0, -23.0, 31.0])
def test_dda_vertical_wall_distance(deg):
    occ = walled(60)
    occ[:, 40] = 1
    a = math.radians(deg)
    t = L.dda_cells(occ, 30, 10, np.float32(math.cos(a)), np.float32(math.sin(a)), 1000.0)
    assert abs(t - (40 - 10.5) / math.cos(a)) < 2e-5 * 40


def test_dda_axis_ray_is_exact_and_grid_edge_is_a_wall():
    occ = np.zeros((20, 30), np.uint8)
    assert L.dda_cells(occ, 5, 3, 1.0, 0.0, 1e3) == 30 - 3.5      # leaves the grid at x = 30
    assert L.dda_cells(occ, 5, 3, 0.0, -1.0, 1e3) == 5.5           # leaves at y = 0
    occ[5, 10] = 1
    assert L.dda_cells(occ, 5, 3, 1.0, 0.0, 1e3) == 6.5
    assert L.dda_cells(occ, 5, 3, 1.0, 0.0, 4.0) == 4.0            # capped at rmax
    assert L.dda_cells(occ, 5, 10, 1.0, 0.0, 1e3) == 0.0           # starts inside an obstacle


def march(occ, j, i, dx, dy, rmax, step=1e-4):
    H, W = occ.shape
    x0, y0 = i + 0.5, j + 0.5
    t = 0.0
    while t < rmax:
        t += step
        ii, jj = math.floor(x0 + t * dx), math.floor(y0 + t * dy)
        if ii < 0 or jj < 0 or ii >= W or jj >= H or occ[jj, ii]:
            return t
    return rmax


def test_dda_matches_fine_march_on_random_grids():
    rng = np.random.default_rng(9)
    checked = 0
    for trial in range(6):
        occ = (rng.random((12, 14)) < 0.2).astype(np.uint8)
        free = np.argwhere(occ == 0)
        for _ in range(20):
            j, i = free[rng.integers(len(free))]
            a = rng.uniform(-math.pi, math.pi)
            dx, dy = np.float32(math.cos(a)), np.float32(math.sin(a))
            t = L.dda_cells(occ, int(j), int(i), dx, dy, 9.0)
            tm = march(occ, int(j), int(i), float(dx), float(dy), 9.0)
            # skip rays that graze a grid vertex (the march then straddles two cells)
            px, py = i + 0.5 + tm * float(dx), j + 0.5 + tm * float(dy)
            if min(abs(px - round(px)), 1) < 1e-3 and abs(py - round(py)) < 1e-3:
                continue
            assert abs(t - tm) < 2e-4, (trial, j, i, a, t, tm)
            checked += 1
    assert checked > 100


# ---------------------------------------------------------------- likelihood + Eq. 9

def test_log_likelihood_closed_form():
    z = np.array([1.0, 2.0, 10.0, 3.0], np.float32)
    r = np.array([[[1.5, 2.0]], [[1.0, 2.1]]], np.float32)   # 2 cells, K=1, stride 2 -> beams 0, 2
    ll = L.log_likelihood(r, z, 10.0, 2, 0.1)
    # beam 2 returned r_max: skipped; only beam 0 counts
    assert abs(ll[0, 0] + 0.25 / 0.02) < 1e-9 and ll[1, 0] == 0.0


def test_reweight_keeps_set_mass_and_leaves_others():
    rng = np.random.default_rng(10)
    b = rng.random((6, 10, 12))
    b /= b.sum()
    cells = np.array([3, 17, 40, 99], np.int32)
    logL = rng.normal(0, 30, (4, 6))
    out = L.reweight(b, cells, logL)
    flat_b, flat_o = b.reshape(6, -1), out.reshape(6, -1)
    others = np.setdiff1d(np.arange(120), cells)
    assert np.array_equal(flat_b[:, others], flat_o[:, others])
    assert abs(flat_o[:, cells].sum() - flat_b[:, cells].sum()) < 1e-15
    assert abs(out.sum() - 1.0) < 1e-14
    # ratios inside the set follow the likelihood ratios (Eq. 9)
    r = (flat_o[:, cells] / flat_b[:, cells]).T
    assert np.allclose(np.log(r / r.max()), logL - logL.max(), atol=1e-9)


def test_reweight_is_the_plain_formula_and_shift_invariant():
    """Eq. 9 normalises L b over the set, so adding a constant to every log-likelihood changes
    nothing.  For moderate values the result equals b w A / sum(b w) with w = exp(log L -
    max log L) written out directly; shifted by -1000 (where that direct form underflows to
    0 / 0) and with the likelihood peaking on zero-belief states, the result is the same."""
    rng = np.random.default_rng(12)
    b = rng.random((5, 9, 11))
    b[:, 2, 3] = 0.0                                 # a sampled cell without belief
    b /= b.sum()
    cells = np.array([5, 2 * 11 + 3, 60, 71], np.int32)
    logL = rng.normal(0, 20, (4, 5))
    logL[1, :] += 60.0                               # the likelihood peaks on the empty cell
    sub = b.reshape(5, -1)[:, cells].T
    w = np.exp(logL - logL.max())
    want = sub * w * (sub.sum() / (sub * w).sum())
    got = L.reweight(b, cells, logL).reshape(5, -1)[:, cells].T
    assert np.allclose(got, want, rtol=1e-12, atol=0.0)
    shifted = L.reweight(b, cells, logL - 1000.0).reshape(5, -1)[:, cells].T
    assert np.allclose(shifted, want, rtol=1e-12, atol=0.0)
    assert np.all(np.isfinite(shifted)) and np.all(shifted[1] == 0.0)


def test_true_pose_scores_best_with_clean_scan():
    """Eq. 10: a noise-free scan from the true state scores at least as high as any other."""
    occ = floorplan.rooms_map(3, size=48)
    cell, K = 0.1, 16
    free = np.argwhere(occ == 0)
    rng = np.random.default_rng(11)
    j, i = free[rng.integers(len(free))]
    k_true = 5
    pose = ((i + 0.5) * cell, (j + 0.5) * cell, 2 * math.pi * k_true / K)
    inc = math.pi / 90
    z = scan.simulate_scan(occ, cell, pose, seed=1, n_beams=180, angle_inc=inc, r_max=3.0,
                           noise_sigma=0.0, dropout=0.0)
    cells = rng.choice(np.flatnonzero(occ.reshape(-1) == 0), 60, replace=False).astype(np.int32)
    cells = np.unique(np.append(cells, j * occ.shape[1] + i)).astype(np.int32)
    ang = L.beam_angles(K, 0.0, 0.0, inc, 180, 2)
    r = L.expected_ranges(occ, cells, L.beam_dirs32(ang), 3.0, cell)
    ll = L.log_likelihood(r, z, 3.0, 2, 0.1)
    c_true = int(np.flatnonzero(cells == j * occ.shape[1] + i)[0])
    assert ll[c_true, k_true] == ll.max()
