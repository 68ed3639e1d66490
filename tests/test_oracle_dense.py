"""Pins of the dense scan update (oracle ``dense``) to facts other than its own formulas: the
range to the grid edge and to walls in closed form, a brute-force fine ray march within half
a code step, the table index against the nearest direction of each beam's absolute angle, the
sampled path's log-likelihood, mass conservation, and Eq. 10 (a clean scan at the true state
scores highest)."""
import math

import numpy as np
import pytest

from oracle import dense as D
from oracle import filter as F
from oracle import lidar as L


def test_range_to_the_grid_edge_along_the_axes():
    H, W, A = 9, 23, 8                       # directions every 45 degrees
    occ = np.zeros((H, W), np.uint8)
    r_max, cell = 40.0, 1.0
    t = D.range_table(occ, A, r_max, cell)
    rmax_cells, inv_step, _ = D.quant(r_max, cell)
    for j in range(H):
        for i in range(W):
            # +x: the walk leaves the grid after W - i - 1/2 cells; +y after H - j - 1/2
            for a, d in ((0, W - i - 0.5), (2, H - j - 0.5), (4, i + 0.5), (6, j + 0.5)):
                want = math.floor(float(np.float32(np.float32(d) * inv_step) + np.float32(0.5)))
                assert t[a, j, i] == min(255, want), (a, j, i)


def test_range_to_a_wall_at_an_angle():
    """A wall column at x = 20: from a cell 8.5 cells to its left, direction phi reaches it
    after 8.5 / cos(phi) cells (the cells crossed before the wall are free)."""
    H, W, A = 41, 30, 36
    occ = np.zeros((H, W), np.uint8)
    occ[:, 20] = 1
    r_max, cell = 60.0, 1.0
    t = D.range_table(occ, A, r_max, cell)
    step = float(np.float32(r_max / 255.0))
    j, i = 20, 11
    for a in (0, 1, 2, 35, 34):
        phi = 2 * math.pi * a / A
        want = (20 - i - 0.5) / abs(math.cos(phi))
        assert abs(t[a, j, i] * step - want) <= step / 2 + 1e-4, (a, t[a, j, i] * step, want)


def test_table_agrees_with_a_fine_ray_march():
    rng = np.random.default_rng(3)
    H, W, A = 24, 31, 24
    occ = (rng.random((H, W)) < 0.12).astype(np.uint8)
    r_max, cell = 12.0, 1.0
    t = D.range_table(occ, A, r_max, cell)
    step = float(np.float32(r_max / 255.0))
    dirs = D.table_dirs32(A).astype(np.float64)
    for _ in range(300):
        j, i, a = int(rng.integers(H)), int(rng.integers(W)), int(rng.integers(A))
        if occ[j, i]:
            assert t[a, j, i] == 0
            continue
        dx, dy = dirs[a]
        x, y, s = i + 0.5, j + 0.5, 0.0
        h = 1e-3
        near_vertex = False          # the walk and the march may pass a lattice vertex apart
        while s < r_max:
            s += h
            px, py = x + s * dx, y + s * dy
            if abs(px - round(px)) < 2e-3 and abs(py - round(py)) < 2e-3:
                near_vertex = True
            ci, cj = math.floor(px), math.floor(py)
            if ci < 0 or ci >= W or cj < 0 or cj >= H or occ[cj, ci]:
                break
        if near_vertex:
            continue
        exact = min(s, r_max)
        assert abs(t[a, j, i] * step - exact) <= step / 2 + 2e-3, (j, i, a, t[a, j, i] * step, exact)


def test_table_index_is_the_nearest_direction_of_the_absolute_beam_angle():
    K, A = 12, 72
    theta, amin, ainc = 0.731, -1.2, 0.0437
    z = np.full(55, 3.0)
    m, zu = D.beam_offsets(theta, amin, ainc, z, 10.0, 2, A)
    bs = list(range(0, 55, 2))
    for k in range(K):
        for n, b in enumerate(bs):
            ang = 2 * math.pi * k / K + theta + amin + ainc * b
            near = round(ang / (2 * math.pi / A)) % A
            assert (k * (A // K) + m[n]) % A == near


def test_log_likelihood_is_the_sampled_models_on_the_tables_ranges():
    rng = np.random.default_rng(5)
    K, A, H, W = 4, 16, 6, 7
    table = rng.integers(0, 256, (A, H, W)).astype(np.uint8)
    z = rng.random(40) * 9.0
    z[5] = 10.0                                            # a dropout, skipped
    r_max, stride, sig = 10.0, 3, 0.2
    m, zu = D.beam_offsets(0.3, -0.5, 0.05, z, r_max, stride, A)
    got = D.log_likelihood(table, K, m, zu, r_max, sig)
    step = float(np.float32(r_max / 255.0))
    # the ranges each state's beams see, then the sampled path's scoring
    used = [b for b in range(0, 40, stride)]
    ranges = np.zeros((H * W, K, len(used)))
    for k in range(K):
        for n, b in enumerate(used):
            x = (0.3 + (-0.5 + 0.05 * b)) / (2 * math.pi / A)
            a = (k * (A // K) + int(math.floor(x + 0.5))) % A
            ranges[:, k, n] = table[a].reshape(-1) * step
    want = L.log_likelihood(ranges, z, r_max, stride, sig)          # (cells, K)
    assert np.abs(got.reshape(K, -1).T - want).max() < 1e-9


def test_update_keeps_mass_zero_walls_and_ignores_dropouts():
    rng = np.random.default_rng(7)
    H, W, K, A = 20, 25, 8, 32
    occ = (rng.random((H, W)) < 0.1).astype(np.uint8)
    f = F.Filter(occ, K, 0.1)
    b = f.B * (1 + rng.random(f.B.shape))
    b /= b.sum()
    table = D.range_table(occ, A, 3.0, 0.1)
    z = rng.random(60) * 3.0
    nb, logL, mx, dl = D.dense_update(b, occ, table, 0.4, z, 0.0, 2 * math.pi / 60, 3.0, 2, 0.1)
    assert abs(nb.sum() - 1.0) < 1e-12 and (nb[:, occ != 0] == 0).all()
    # every beam a dropout: nothing changes and the normaliser is 1
    nb2, _, _, dl2 = D.dense_update(b, occ, table, 0.4, np.full(60, 3.0), 0.0, 0.1, 3.0, 2, 0.1)
    assert np.abs(nb2 - b).max() < 1e-15 and abs(dl2) < 1e-12
    # the normaliser: log(sum b w) + max, with w = exp(logL - max)
    w = np.exp(logL - mx) * (occ == 0)
    assert abs(dl - (math.log((b * w).sum()) + mx)) < 1e-9


def test_a_clean_scan_on_the_table_grid_scores_the_true_state_highest():
    """Eq. 10: ranges read off the table at the true state (beams on the table directions)
    give log L = 0 there, the maximum, so the true state gains the most."""
    rng = np.random.default_rng(11)
    H, W, K, A = 30, 30, 12, 72
    occ = np.zeros((H, W), np.uint8)
    occ[0, :] = occ[-1, :] = occ[:, 0] = occ[:, -1] = 1
    occ[8:12, 17:20] = 1
    occ[20, 5:14] = 1
    r_max, cell = 2.5, 0.1
    table = D.range_table(occ, A, r_max, cell)
    step = float(np.float32(r_max / 255.0))
    kt, jt, it = 5, 14, 9
    n = A                                                   # one beam per table direction
    ainc = 2 * math.pi / A
    z = np.array([table[(kt * (A // K) + b) % A, jt, it] * step for b in range(n)])
    z = np.minimum(z, r_max - 1e-9)
    f = F.Filter(occ, K, cell)
    nb, logL, mx, _ = D.dense_update(f.B, occ, table, 0.0, z, 0.0, ainc, r_max, 1, 0.05)
    assert logL[kt, jt, it] == pytest.approx(0.0, abs=1e-9) and mx == pytest.approx(0.0, abs=1e-9)
    assert nb[kt, jt, it] == nb.max()


def test_map_difficulty_of_a_featureless_corridor():
    """A corridor much longer than r_max: along its middle every cell sees the same scan (the
    side walls; the beams along the corridor are capped and skipped, like dropouts), so the best
    match of a probe there is the first cell of its row that agrees with the probe on every used
    beam, and the error is the distance to it."""
    H, W, K, A = 7, 80, 4, 16
    occ = np.zeros((H, W), np.uint8)
    occ[0, :] = occ[-1, :] = 1
    cell, r_max = 0.1, 1.0                                   # r_max = 10 cells << 80
    table = D.range_table(occ, A, r_max, cell)
    probes = np.array([3 * W + i for i in (20, 30, 40, 50, 60)])
    e, n = D.map_difficulty(occ, table, K, cell, r_max, probes, 0, 1, 0.1, 1.0)
    # the probe's used directions (code < 255 in its own column), and the first cell of row 3
    # (bin 0) whose codes agree on all of them
    used = [a for a in range(A) if table[a, 3, 40] < 255]
    first = next(i for i in range(W) if all(table[a, 3, i] == table[a, 3, 40] for a in used))
    assert 0 < first < 20
    assert np.allclose(e, [cell * (i - first) for i in (20, 30, 40, 50, 60)])
    assert n == 5                                            # all farther than 1 m


def test_map_difficulty_is_zero_where_every_scan_is_distinct():
    """Noise-free probes in a room with distinct features: each probe's own state matches
    exactly (log L = 0) and no other free state within the cap does, so e_p = 0."""
    rng = np.random.default_rng(2)
    H, W, K, A = 20, 26, 8, 32
    occ = np.zeros((H, W), np.uint8)
    occ[0, :] = occ[-1, :] = occ[:, 0] = occ[:, -1] = 1
    occ[5:7, 8:10] = 1
    occ[12, 15:20] = 1
    occ[3:9, 19] = 1
    cell, r_max = 0.1, 3.0
    table = D.range_table(occ, A, r_max, cell)
    free = np.flatnonzero(occ.reshape(-1) == 0)
    probes = rng.choice(free, 25, replace=False)
    e, n = D.map_difficulty(occ, table, K, cell, r_max, probes, 0, 1, 0.1, 1.0)
    assert n == 0 and e.max() == 0.0


def test_map_difficulty_of_two_identical_rooms_finds_the_copy():
    """Two closed rooms, one a translate of the other: the walk depends only on offsets, so a
    probe in the second room (the larger index) sees exactly the scan of its copy in the first,
    and the tie goes to the copy; a probe in the first room matches itself."""
    H, W, K, A = 12, 40, 8, 32
    occ = np.zeros((H, W), np.uint8)
    occ[0, :] = occ[-1, :] = 1
    occ[:, 0] = occ[:, 19] = occ[:, 20] = occ[:, 39] = 1
    occ[3, 5] = occ[3, 25] = 1                               # the same feature in both rooms
    occ[8, 12:15] = occ[8, 32:35] = 1
    cell, r_max = 0.1, 3.0
    table = D.range_table(occ, A, r_max, cell)
    probes = np.array([6 * W + 8, 6 * W + 28])
    e, n = D.map_difficulty(occ, table, K, cell, r_max, probes, 0, 1, 0.1, 1.0)
    assert e[0] == 0.0 and abs(e[1] - 2.0) < 1e-12 and n == 1
