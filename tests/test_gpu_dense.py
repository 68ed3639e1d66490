"""GPU parity of the dense scan update (Eq. 9 on every state from the expected-range table)
through the C-ABI against the oracle ``oracle.dense``.

* The table: bit-exact (the same FP32 grid walk and quantisation operations, no contraction).
* The update, FP32 storage: the GPU scores in FP32.  Each state's log-likelihood carries at most
  about (n_used + 8) 2^-23 (|log L| + 1) of rounding, and the update divides by exp(max log L).
  So a state's relative error is bounded by (n_used + 8) 2^-23 (|log L| + |max log L| + 2),
  plus 2^-20 for the normalisation and storage.  The test checks every state against that
  bound, computed from the oracle's own log L, and against the 1e-6 absolute bar.
* Reduced precision: L1 <= 1e-2 and the same argmax wherever the oracle's maximum is
  unambiguous.
"""
import math

import numpy as np
import pytest

import paper_1910_00572_gb300 as loc
from oracle import dense as D
from oracle import filter as F
from oracle import readout as R
from synth import fields, floorplan, scan, trajectory

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1910_00572_gb300 import build
    build.build()
    loc.lib()


def make(occ, K, cell, **kw):
    p = loc.loc_params_default(H=occ.shape[0], W=occ.shape[1], K=K, cell_m=cell, **kw)
    return loc.loc_create(occ, p)


def bound(ref, logL, mx, n_used):
    """Per-state error bound of the FP32 update (module docstring)."""
    rel = (n_used + 8) * 2.0 ** -23 * (np.abs(logL) + abs(mx) + 2.0) + 2.0 ** -20
    return np.where(np.isfinite(rel), rel, 0.0) * ref + 1e-12


def check_update(got, ref, logL, mx, n_used):
    err = np.abs(got.astype(np.float64) - ref)
    assert err.max() <= 1e-6, err.max()
    tol = bound(ref, logL, mx, n_used)
    worst = (err / tol).max()
    assert worst <= 1.0, worst
    return float(err.max())


@pytest.mark.parametrize("H,W,K,A", [(37, 53, 12, 72), (64, 64, 16, 64), (40, 44, 8, 8)],
                         ids=["ragged, 6 directions per bin", "tile-aligned", "one direction per bin"])
def test_table_is_bit_exact(H, W, K, A):
    occ = floorplan.rooms_map(3, size=max(H, W))[:H, :W].copy()
    cell, r_max = 0.1, 2.5
    h = make(occ, K, cell)
    try:
        loc.loc_range_table(h, A, r_max)
        got = loc.loc_range_table_read(h)
    finally:
        loc.loc_destroy(h)
    want = D.range_table(occ, A, r_max, cell)
    assert np.array_equal(got, want), np.argwhere(got != want)[:5]


def scan_at(occ, cell, pose, seed, n_beams=360, r_max=2.5):
    return scan.simulate_scan(occ, cell, pose, seed=seed, n_beams=n_beams, angle_min=-math.pi,
                              angle_inc=2 * math.pi / n_beams, r_max=r_max, noise_sigma=0.03,
                              dropout=0.05, march=0.25)


@pytest.mark.parametrize("H,W,K,A,stride", [(48, 61, 12, 72, 4), (64, 64, 16, 128, 3), (33, 40, 20, 120, 8)],
                         ids=["ragged", "tile-aligned, 16 bins", "K not a multiple of 16"])
def test_update_matches_oracle(H, W, K, A, stride):
    occ = floorplan.rooms_map(9, size=max(H, W))[:H, :W].copy()
    cell, r_max, sig = 0.1, 2.5, 0.1
    b0 = fields.belief_like(occ, K, seed=H + K, dtype=np.float32)
    ref_b = b0.astype(np.float64) / b0.astype(np.float64).sum()
    free = np.argwhere(occ == 0)
    j, i = free[len(free) // 2]
    z = scan_at(occ, cell, ((i + 0.5) * cell, (j + 0.5) * cell, 0.7), seed=H)
    h = make(occ, K, cell)
    try:
        loc.loc_set_belief(h, b0)
        loc.loc_range_table(h, A, r_max)
        st0 = loc.loc_stats(h)
        loc.loc_lidar_update_dense(h, z, -math.pi, 2 * math.pi / len(z), stride, sig)
        got = loc.loc_belief(h)
        st = loc.loc_stats(h)
    finally:
        loc.loc_destroy(h)
    table = D.range_table(occ, A, r_max, cell)
    nb, logL, mx, dl = D.dense_update(ref_b, occ, table, 0.0, z, -math.pi, 2 * math.pi / len(z), r_max,
                                      stride, sig)
    n_used = int(((z[::stride]) < r_max).sum())
    check_update(got, nb, logL, mx, n_used)
    assert (got[:, occ != 0] == 0).all()
    assert abs((st["logscale"] - st0["logscale"]) - dl) <= 1e-5 * max(1.0, abs(dl))


def test_scans_and_steps_follow_the_oracle():
    """A walk with a dense scan every fourth step: propagation and the dense update alternate
    on the same session."""
    occ = floorplan.rooms_map(12, size=56)
    K, cell, r_max, sig, A, stride = 16, 0.1, 2.5, 0.1, 64, 6
    walk = trajectory.random_walk(occ, cell, 16, 0.1, 21)
    h = make(occ, K, cell)
    f = F.Filter(occ, K, cell)
    ref = D.Filter(f, occ, cell, A, r_max)
    try:
        loc.loc_range_table(h, A, r_max)
        for t, (u, v, w) in enumerate(walk.odom, start=1):
            loc.loc_step(h, u, v, w)
            f.step(u, v, w)
            if t % 4 == 0:
                z = scan_at(occ, cell, walk.poses[t], seed=100 + t)
                loc.loc_lidar_update_dense(h, z, -math.pi, 2 * math.pi / len(z), stride, sig)
                ref.dense_update(z, -math.pi, 2 * math.pi / len(z), stride, sig)
                got = loc.loc_belief(h)
                err = np.abs(got.astype(np.float64) - f.B)
                # the step errors (1e-6 bar) carry through the weights; the scan adds its own bound
                assert err.max() <= 1e-6, (t, err.max())
                assert np.abs(got.astype(np.float64) - f.B).sum() <= 1e-4, t
        st = loc.loc_stats(h)
        assert abs(st["logscale"] - f.logscale) <= 1e-4 * max(1.0, abs(f.logscale))
        k, j, i, _ = R.argmax_pose(f.B)
        top2 = np.sort(f.B.reshape(-1))[-2:]
        if top2[1] - top2[0] > 2e-2 * top2[1]:
            assert loc.loc_argmax(h)[:3] == (k, j, i)
    finally:
        loc.loc_destroy(h)


@pytest.mark.parametrize("storage", ["bf16", "f16"])
def test_reduced_precision_l1_and_argmax(storage):
    occ = floorplan.rooms_map(14, size=64)
    K, cell, r_max, sig, A, stride = 16, 0.1, 2.5, 0.1, 64, 4
    walk = trajectory.random_walk(occ, cell, 12, 0.1, 5)
    h = make(occ, K, cell, storage=storage)
    f = F.Filter(occ, K, cell)
    ref = D.Filter(f, occ, cell, A, r_max)
    try:
        loc.loc_range_table(h, A, r_max)
        for t, (u, v, w) in enumerate(walk.odom, start=1):
            loc.loc_step(h, u, v, w)
            f.step(u, v, w)
            if t % 3 == 0:
                z = scan_at(occ, cell, walk.poses[t], seed=200 + t)
                loc.loc_lidar_update_dense(h, z, -math.pi, 2 * math.pi / len(z), stride, sig)
                ref.dense_update(z, -math.pi, 2 * math.pi / len(z), stride, sig)
                b = loc.loc_belief(h).astype(np.float64)
                assert np.abs(b - f.B).sum() <= 1e-2, t
                k, j, i, _ = R.argmax_pose(f.B)
                top2 = np.sort(f.B.reshape(-1))[-2:]
                if top2[1] - top2[0] > 2e-2 * top2[1]:
                    assert loc.loc_argmax(h)[:3] == (k, j, i), t
    finally:
        loc.loc_destroy(h)


def test_dropouts_change_nothing_and_the_restart_state_is_scored():
    occ = floorplan.rooms_map(15, size=40)
    K, cell, r_max, A = 8, 0.1, 2.5, 64
    h = make(occ, K, cell)
    try:
        loc.loc_range_table(h, A, r_max)
        before = loc.loc_belief(h)                        # the restart state: uniform
        loc.loc_lidar_update_dense(h, np.full(90, r_max, np.float32), 0.0, 0.07, 1, 0.1)
        assert np.array_equal(loc.loc_belief(h), before)
        z = scan_at(occ, cell, (2.05, 1.95, 0.3), seed=3)
        loc.loc_lidar_update_dense(h, z, -math.pi, 2 * math.pi / len(z), 5, 0.1)
        got = loc.loc_belief(h)
    finally:
        loc.loc_destroy(h)
    M = (occ == 0).astype(np.float64)
    table = D.range_table(occ, A, r_max, cell)
    nb, logL, mx, _ = D.dense_update(F.uniform_belief(M, K), occ, table, 0.0, z, -math.pi,
                                     2 * math.pi / len(z), r_max, 5, 0.1)
    check_update(got, nb, logL, mx, int((z[::5] < r_max).sum()))


def test_arguments_are_checked():
    occ = floorplan.rooms_map(16, size=32)
    h = make(occ, 8, 0.1)
    try:
        z = np.full(10, 1.0, np.float32)
        with pytest.raises(loc.LocError) as e:
            loc.loc_lidar_update_dense(h, z, 0.0, 0.1, 1, 0.1)      # no table yet
        assert e.value.status == loc.LOC_ERR_INVALID_ARG
        for A in (0, 12, 8 * 181):                                   # not a multiple of K / too many
            with pytest.raises(loc.LocError):
                loc.loc_range_table(h, A, 2.0)
        with pytest.raises(loc.LocError):
            loc.loc_range_table(h, 64, -1.0)
        loc.loc_range_table(h, 64, 2.0)
        with pytest.raises(loc.LocError):
            loc.loc_lidar_update_dense(h, np.full(3000, 1.0, np.float32), 0.0, 0.001, 1, 0.1)
        with pytest.raises(loc.LocError):
            loc.loc_lidar_update_dense(h, np.array([1.0, np.nan], np.float32), 0.0, 0.1, 1, 0.1)
        assert loc.loc_stats(h)["n_propagations"] == 0
    finally:
        loc.loc_destroy(h)


def map_cases():
    H, W = 7, 80                                        # a featureless corridor
    corridor = np.zeros((H, W), np.uint8)
    corridor[0, :] = corridor[-1, :] = 1
    rooms = np.zeros((12, 40), np.uint8)                 # two identical closed rooms
    rooms[0, :] = rooms[-1, :] = 1
    rooms[:, 0] = rooms[:, 19] = rooms[:, 20] = rooms[:, 39] = 1
    rooms[3, 5] = rooms[3, 25] = 1
    rooms[8, 12:15] = rooms[8, 32:35] = 1
    plan = floorplan.rooms_map(21, size=48)[:45, :47].copy()
    return [("corridor", corridor, 4, 16, 1.0, [3 * 80 + i for i in (5, 20, 40, 60, 78)]),
            ("two rooms", rooms, 8, 32, 3.0, [6 * 40 + 8, 6 * 40 + 28, 2 * 40 + 2, 9 * 40 + 37]),
            ("rooms plan", plan, 8, 64, 2.0, None)]


@pytest.mark.parametrize("case", range(3), ids=["corridor", "two rooms", "rooms plan"])
@pytest.mark.parametrize("probe_bin,beam_step", [(0, 1), (3, 2)])
def test_map_difficulty_matches_oracle(case, probe_bin, beam_step):
    name, occ, K, A, r_max, probes = map_cases()[case]
    cell = 0.1
    if probes is None:
        free = np.flatnonzero(occ.reshape(-1) == 0)
        probes = np.random.default_rng(4).choice(free, 40, replace=False)
    probes = np.asarray(probes, np.int32)
    h = make(occ, K, cell)
    try:
        loc.loc_range_table(h, A, r_max)
        got_e, got_n = loc.loc_map_difficulty(h, probes, probe_bin, beam_step, 0.1, 1.0)
        b_after = loc.loc_belief(h)
        assert np.array_equal(b_after, loc.loc_belief(h))
    finally:
        loc.loc_destroy(h)
    table = D.range_table(occ, A, r_max, cell)
    want_e, want_n = D.map_difficulty(occ, table, K, cell, r_max, probes, probe_bin, beam_step, 0.1, 1.0)
    assert np.abs(got_e - want_e).max() <= 1e-9, (name, got_e, want_e)
    assert got_n == want_n


def test_map_difficulty_arguments():
    occ = floorplan.rooms_map(22, size=32)
    h = make(occ, 8, 0.1)
    try:
        free = int(np.flatnonzero(occ.reshape(-1) == 0)[0])
        wall = int(np.flatnonzero(occ.reshape(-1) != 0)[0])
        with pytest.raises(loc.LocError):
            loc.loc_map_difficulty(h, [free], 0, 1, 0.1, 1.0)            # no table
        loc.loc_range_table(h, 32, 2.0)
        with pytest.raises(loc.LocError) as e:
            loc.loc_map_difficulty(h, [free, wall], 0, 1, 0.1, 1.0)      # an occupied probe
        assert "occupied" in loc.loc_last_error(h)
        for bad in (dict(probe_bin=8), dict(beam_step=0), dict(sigma_r=0.0), dict(c_m=-1.0)):
            kw = dict(probe_bin=0, beam_step=1, sigma_r=0.1, c_m=1.0)
            kw.update(bad)
            with pytest.raises(loc.LocError):
                loc.loc_map_difficulty(h, [free], **kw)
        with pytest.raises(loc.LocError):
            loc.loc_map_difficulty(h, [32 * 32], 0, 1, 0.1, 1.0)       # out of the grid
        e, n = loc.loc_map_difficulty(h, [free], 0, 1, 0.1, 1.0)
        assert e.shape == (1,) and n in (0, 1)
    finally:
        loc.loc_destroy(h)
