"""GPU parity of the propagation (Alg. 1 + Eq. 9) through the C-ABI against the FP64 oracle.

Tolerances (FP32 storage): the normalised belief agrees to 1e-6 absolute (the stated bar) and
to 2e-5 of the tensor's maximum (derived: one step rounds ~1 + 4 + 5 + 5 + 7 + 2 FP32 terms per
output, each a relative 2^-24, so a step adds well under 1e-5 relative; the map correction and
the blur contract older errors).  Integer-shift permutations are bit-exact.
"""
import math

import numpy as np
import pytest

import bounds
import paper_1910_00572_gb300 as loc
from oracle import filter as F
from oracle import readout as R
from oracle.odometry import Odometry
from synth import fields, floorplan, workloads

pytestmark = pytest.mark.gpu

ABS_TOL = 1e-6
REL_TOL = 2e-5


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1910_00572_gb300 import build
    build.build()
    loc.lib()


def make(occ, K, cell, **kw):
    p = loc.loc_params_default(H=occ.shape[0], W=occ.shape[1], K=K, cell_m=cell, **kw)
    return loc.loc_create(occ, p)


def check_close(gpu, ref, abs_tol=ABS_TOL, rel_tol=REL_TOL):
    err = np.abs(gpu.astype(np.float64) - ref)
    assert err.max() <= abs_tol, err.max()
    assert err.max() <= rel_tol * ref.max(), (err.max(), ref.max())
    return float(err.max())


# ------------------------------------------------------------------ full trajectory, small grid

@pytest.fixture(scope="module")
def rooms64_run():
    wl = workloads.get("rooms64")
    occ = workloads.make_map(wl)
    walk = workloads.make_walk(wl, occ)
    checkpoints = {1, 2, 10, 50, 100, 200}
    h = make(occ, wl["K"], wl["cell"])
    ref = F.Filter(occ, wl["K"], wl["cell"], wl["sigma_xy_cells"], wl["sigma_theta_bins"])
    out = []
    try:
        for t, (u, v, w) in enumerate(walk.odom, start=1):
            assert loc.loc_step(h, u, v, w) == loc.LOC_OK
            ref.step(u, v, w)
            if t in checkpoints:
                st = loc.loc_stats(h)
                out.append((t, loc.loc_belief(h), ref.B.copy(), st, ref.last_Z, ref.logscale,
                            loc.loc_argmax(h), loc.loc_marginal(h, loc.LOC_MAP_MAX)))
    finally:
        loc.loc_destroy(h)
    return occ, out


def test_rooms64_trajectory_matches_oracle(rooms64_run):
    _, out = rooms64_run
    for t, b, rb, st, Z, ls, _, _ in out:
        check_close(b, rb)
        assert abs(st["last_Z"] - Z) <= 1e-6 * Z, (t, st["last_Z"], Z)
        assert abs(st["logscale"] - ls) <= 1e-5 * max(1.0, abs(ls)), (t, st["logscale"], ls)
        assert st["n_propagations"] == t


def test_rooms64_occupied_cells_hold_no_mass(rooms64_run):
    occ, out = rooms64_run
    for _, b, *_ in out:
        assert (b[:, occ != 0] == 0.0).all()


def test_rooms64_estimate_and_belief_map(rooms64_run):
    _, out = rooms64_run
    for t, b, rb, _, _, _, am, m in out:
        k, j, i, p = R.argmax_pose(rb)
        top2 = np.sort(rb.reshape(-1))[-2:]
        if top2[1] - top2[0] > 2 * ABS_TOL:            # unambiguous maximum
            assert am[:3] == (k, j, i), (t, am, (k, j, i))
        assert abs(am[3] - p) <= ABS_TOL
        check_close(m, R.belief_map(rb, "max"))


# ------------------------------------------------------------------ exact cases

def test_zero_noise_integer_shift_is_bit_exact_permutation():
    H, W, K = 40, 72, 4
    occ = np.zeros((H, W), np.uint8)
    rng = np.random.default_rng(0)
    b = np.zeros((K, H, W))
    b[:, 12:28, 20:52] = rng.integers(1, 64, (K, 16, 32))
    b = (b / b.sum() * 2 ** 20).round()
    b[0, 12, 20] += 2 ** 20 - b.sum()                  # sum exactly 2^20
    b = (b / 2 ** 20).astype(np.float32)               # values k / 2^20, sum exactly 1
    h = make(occ, K, 1.0, sigma_xy_cells=0.0, sigma_theta_bins=0.0)
    try:
        loc.loc_set_belief(h, b)
        loc.loc_step(h, 3.0, 0.0, 0.0)                 # 3 cells along each channel's heading
        got = loc.loc_belief(h)
        assert loc.loc_stats(h)["last_Z"] == 1.0
    finally:
        loc.loc_destroy(h)
    want = np.stack([np.roll(b[0], 3, 1), np.roll(b[1], 3, 0),
                     np.roll(b[2], -3, 1), np.roll(b[3], -3, 0)])
    assert np.array_equal(got, want)


def test_mass_is_conserved_on_a_free_map():
    occ = np.zeros((96, 96), np.uint8)
    b = np.zeros((8, 96, 96), np.float32)
    b[:, 30:66, 30:66] = np.random.default_rng(1).random((8, 36, 36))
    h = make(occ, 8, 0.05)
    try:
        loc.loc_set_belief(h, b)
        for _ in range(3):
            loc.loc_step(h, 0.071, -0.043, 0.02)       # 1.4 / 0.9 cells per step
            assert abs(loc.loc_stats(h)["last_Z"] - 1.0) < 1e-6
    finally:
        loc.loc_destroy(h)


def test_uniform_belief_is_a_fixed_point_at_walls():
    """Algorithm 1's edge correction ('wall, not cliff'): zero motion keeps the uniform belief uniform."""
    occ = floorplan.rooms_map(5, size=64)
    h = make(occ, 8, 0.1)
    try:
        b0 = loc.loc_belief(h)
        loc.loc_step(h, 0.0, 0.0, 0.0)
        b1 = loc.loc_belief(h)
    finally:
        loc.loc_destroy(h)
    assert np.abs(b1 - b0).max() <= 1e-6 * b0.max()


# ------------------------------------------------------------------ edge cases vs the oracle

CASES = [
    # (H, W, K, sigma_xy, sigma_theta, motion (u, v, w) in cells/rad, label)
    (37, 53, 5, 0.5, 1.0, (0.4, -1.3, 0.1), "ragged tiles"),
    (1, 70, 3, 0.5, 1.0, (2.2, 0.0, 0.0), "single row, K < theta kernel"),
    (70, 1, 2, 0.5, 1.0, (0.0, 1.6, 0.0), "single column"),
    (17, 33, 1, 0.5, 1.0, (0.25, 0.75, 0.0), "one bin"),
    (48, 48, 12, 0.9, 1.3, (-0.6, 0.35, -0.2), "radii 3 / 4"),
    (33, 65, 6, 0.0, 0.0, (0.5, 0.5, 0.0), "zero noise, half-cell shift"),
    (40, 40, 4, 0.5, 1.0, (25.3, -14.6, 0.0), "shift beyond the tile"),
]


@pytest.mark.parametrize("H,W,K,sxy,sth,mot,label", CASES, ids=[c[-1] for c in CASES])
def test_edge_cases_match_oracle(H, W, K, sxy, sth, mot, label):
    rng = np.random.default_rng(H * 1000 + W)
    occ = (rng.random((H, W)) < 0.15).astype(np.uint8)
    occ[H // 2, W // 2] = 0
    cell = 0.1
    b = fields.belief_like(occ, K, seed=H + W, dtype=np.float32)
    h = make(occ, K, cell, sigma_xy_cells=sxy, sigma_theta_bins=sth)
    ref = F.Filter(occ, K, cell, sxy, sth)
    ref.B = b.astype(np.float64) / b.astype(np.float64).sum()
    try:
        loc.loc_set_belief(h, b)
        for _ in range(2):
            u, v, w = mot[0] * cell, mot[1] * cell, mot[2]
            loc.loc_step(h, u, v, w)
            ref.step(u, v, w)
            if ref.last_Z == 0.0:
                break
            check_close(loc.loc_belief(h), ref.B)
    finally:
        loc.loc_destroy(h)


def test_all_mass_removed_restarts_uniform():
    occ = np.ones((24, 24), np.uint8)
    occ[10:14, 10:14] = 0
    h = make(occ, 2, 1.0, sigma_xy_cells=0.0, sigma_theta_bins=0.0)
    try:
        loc.loc_step(h, 6.0, 0.0, 0.0)                 # every hypothesis walks into a wall
        assert loc.loc_sync(h) == loc.LOC_WARN_REINIT   # reported once ...
        assert loc.loc_sync(h) == loc.LOC_OK            # ... per new restart
        st = loc.loc_stats(h)
        b = loc.loc_belief(h)
        loc.loc_step(h, 6.0, 0.0, 0.0)                 # the uniform restart walks into the walls again
        assert loc.loc_sync(h) == loc.LOC_WARN_REINIT
        assert loc.loc_stats(h)["n_reinit"] == 2
    finally:
        loc.loc_destroy(h)
    assert st["n_reinit"] == 1 and st["last_Z"] == 0.0
    M = (occ == 0).astype(np.float64)
    assert np.abs(b - F.uniform_belief(M, 2)).max() <= 1e-9


def test_gate_defers_until_one_cell():
    occ = floorplan.rooms_map(2, size=64)
    h = make(occ, 8, 0.1, min_shift_cells=1.0)
    ref = F.Filter(occ, 8, 0.1, min_shift_cells=1.0)
    try:
        for (u, v, w) in [(0.03, 0.0, 0.05), (0.04, 0.01, 0.1), (0.05, 0.0, 0.0)]:
            s = loc.loc_step(h, u, v, w)
            moved = ref.step(u, v, w)
            assert s == (loc.LOC_OK if moved else loc.LOC_OK_DEFERRED)
        assert ref.n_prop == 1
        check_close(loc.loc_belief(h), ref.B)
        assert abs(loc.loc_stats(h)["theta"] - ref.odo.theta) < 1e-15
    finally:
        loc.loc_destroy(h)


def test_invalid_odometry_is_rejected_without_state_change():
    occ = floorplan.rooms_map(2, size=64)
    h = make(occ, 4, 0.1)
    try:
        with pytest.raises(loc.LocError) as e:
            loc.loc_step(h, float("nan"), 0.0, 0.0)
        assert e.value.status == loc.LOC_ERR_INVALID_ARG
        st = loc.loc_stats(h)
        assert st["n_propagations"] == 0 and st["theta"] == 0.0
    finally:
        loc.loc_destroy(h)


def test_steps_are_deterministic():
    occ = floorplan.rooms_map(4, size=64)
    outs = []
    for _ in range(2):
        h = make(occ, 16, 0.1)
        try:
            for t in range(5):
                loc.loc_step(h, 0.037 * t, -0.02, 0.03)
            outs.append((loc.loc_belief(h), loc.loc_stats(h)["last_Z"]))
        finally:
            loc.loc_destroy(h)
    assert np.array_equal(outs[0][0], outs[1][0]) and outs[0][1] == outs[1][1]


# ------------------------------------------------------------------ full-size one-step replay

def test_office512_one_step_replay_sampled():
    wl = workloads.get("office512")
    occ = workloads.make_map(wl)
    K, cell = wl["K"], wl["cell"]
    b32 = fields.belief_like(occ, K, seed=11, dtype=np.float32)
    h = make(occ, K, cell)
    u, v, w = 0.0123, -0.0071, 0.004
    try:
        loc.loc_set_belief(h, b32)
        loc.loc_step(h, u, v, w)
        got = loc.loc_belief(h)
        Z = loc.loc_stats(h)["last_Z"]
    finally:
        loc.loc_destroy(h)
    b_in = b32.astype(np.float64)
    b_in /= b_in.sum()
    odo = Odometry(K, cell)
    odo.add(u, v, w)
    M = F.traversability(occ)
    g = F.motion_kernel(wl["sigma_xy_cells"], wl["sigma_theta_bins"])
    rng = np.random.default_rng(5)
    H, W = occ.shape
    idx = [(int(rng.integers(K)), int(rng.integers(H)), int(rng.integers(W))) for _ in range(1500)]
    # include the states around the largest input values (sharp peaks)
    for q in np.argsort(b_in.reshape(-1))[-20:]:
        k, rem = divmod(int(q), H * W)
        idx.append((k, rem // W, rem % W))
    T = F.propagate_at(b_in, M, odo.shifts(), g, idx)
    gotT = np.array([got[k, j, i] for (k, j, i) in idx], np.float64) * Z
    err = np.abs(gotT - T)
    assert err.max() <= ABS_TOL and err.max() <= REL_TOL * b_in.max(), err.max()
    # Z is the FP64 sum of the stored tensor (a property at any size)
    assert abs(got.astype(np.float64).sum() - 1.0) < 1e-5


@pytest.mark.slow
def test_office2048_bf16_one_step_replay_sampled():
    """The 2048 x 2048 x 72 BF16 office workload at full size (302 M states), one step through
    the tile configuration the benchmark times (the session default): 3000 random states, the
    neighbourhoods of the ten largest input values, and the GPU's argmax state, each recomputed
    from the definitions by the oracle from the same stored input.  Every state is within one
    BF16 rounding step of its own exact value plus the FP32 error (tests/bounds.py),
    the argmax state holds at least every checked state's value, and the tensor sums to 1."""
    wl = workloads.get("office2048")
    occ = workloads.make_map(wl)
    K, cell = wl["K"], wl["cell"]
    H, W = occ.shape
    h = make(occ, K, cell, storage="bf16")
    u, v, w = 0.0137, -0.0061, 0.003
    try:
        loc.loc_set_belief(h, fields.belief_like(occ, K, seed=21, dtype=np.float32))
        before = loc.loc_belief(h)                      # the stored BF16 input, normalised
        loc.loc_step(h, u, v, w)
        got = loc.loc_belief(h)
        Z = loc.loc_stats(h)["last_Z"]
        ak, aj, ai, _ = loc.loc_argmax(h)
    finally:
        loc.loc_destroy(h)
    odo = Odometry(K, cell)
    odo.add(u, v, w)
    M = F.traversability(occ)
    g = F.motion_kernel(wl["sigma_xy_cells"], wl["sigma_theta_bins"])
    rng = np.random.default_rng(8)
    idx = [(int(rng.integers(K)), int(rng.integers(H)), int(rng.integers(W))) for _ in range(3000)]
    for q in np.argpartition(before.reshape(-1), -10)[-10:]:
        k, rem = divmod(int(q), H * W)
        j, i = rem // W, rem % W
        idx += [(k, jj, ii) for jj in range(max(0, j - 2), min(H, j + 3)) for ii in range(max(0, i - 2), min(W, i + 3))]
    idx.append((ak, aj, ai))
    T = F.propagate_at(before.astype(np.float64), M, odo.shifts(), g, idx)
    gotT = np.array([got[k, j, i] for (k, j, i) in idx], np.float64) * Z
    bound = bounds.bf16_step_bound(T)
    bad = np.flatnonzero(np.abs(gotT - T) > bound)
    assert bad.size == 0, [(idx[b], gotT[b], T[b], bound[b]) for b in bad[:5]]
    assert T[-1] >= T.max() - 2.0 * bounds.bf16_step_bound(T.max())
    assert abs(got.astype(np.float64).sum() - 1.0) < 1e-4


@pytest.mark.parametrize("tile,kernel", [(3, "tiled"), (6, "tiled"), (16, "tiled"), (8, "tiled"), (0, "generic")])
def test_bf16_rounding_keeps_each_cells_theta_mass(tile, kernel):
    """BF16 stores round by error diffusion along theta: each stored value is one of the two BF16
    neighbours of its value (within one unit in the last place of its exact value, plus the FP32
    error), and the residual a cell carries from plane to plane keeps the cell's total over its
    bins: |sum_k stored - sum_k exact| <= half a unit in the last place of the cell's largest
    value, plus the FP32 error.  (The residual never grows: a plane either absorbs it within
    half a unit of its own value or passes on less of it.)  Independent rounding of each value,
    stochastic or to nearest, misses the second bound on cells whose bins hold several values of
    similar size, since its error sums grow like the square root of their number.  Synchronous,
    warp-specialised, paired and generic kernels alike."""
    from oracle import cprop
    occ = floorplan.crop(floorplan.office_map(5, size=256), 40, 30, 96, 128)
    K, cell = 72, 0.05
    kw = dict(tile=tile) if kernel == "tiled" else dict(kernel=loc.LOC_KERNEL_GENERIC)
    h = make(occ, K, cell, storage="bf16", **kw)
    u, v, w = 0.0137, -0.0061, 0.0
    try:
        loc.loc_set_belief(h, fields.belief_like(occ, K, seed=4, dtype=np.float32))
        before = loc.loc_belief(h).astype(np.float64)          # the stored BF16 input, normalised
        loc.loc_step(h, u, v, w)
        got = loc.loc_belief(h).astype(np.float64) * loc.loc_stats(h)["last_Z"]
    finally:
        loc.loc_destroy(h)
    odo = Odometry(K, cell)
    odo.add(u, v, w)
    M = F.traversability(occ)
    g = F.motion_kernel(0.5, 1.0)
    T = cprop.propagate(before, M, F.edge_correction(M, K, g), odo.shifts(), g, cprop.host_cores())
    bad = np.flatnonzero(np.abs(got - T) > bounds.bf16_step_bound(T))
    assert bad.size == 0, bad[:5]
    cell_err = np.abs(got.sum(axis=0) - T.sum(axis=0))
    cell_bound = 0.5 * bounds.bf16_ulp(T.max(axis=0) * (1.0 + 1e-5)) + 5e-6 * T.sum(axis=0)
    worst = np.unravel_index(np.argmax(cell_err - cell_bound), cell_err.shape)
    assert np.all(cell_err <= cell_bound), (worst, cell_err[worst], cell_bound[worst])


@pytest.mark.parametrize("storage", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("H,W,K", [(16, 24, 8), (7, 9, 3)])
def test_argmax_ties_restart_and_ragged_sizes(storage, H, W, K):
    """loc_argmax: the most probable state with ties going to the lowest [K][H][W] index, the
    uniform restart state (first free cell of bin 0), and element counts that are not a
    multiple of the vector width (7 x 9 x 3)."""
    occ = np.zeros((H, W), np.uint8)
    occ[0, :2] = 1                                    # the first free cell is (0, 0, 2)
    p = loc.loc_params_default(H=H, W=W, K=K, cell_m=0.1, storage=storage)
    h = loc.loc_create(occ, p)
    try:
        k, j, i, pr = loc.loc_argmax(h)                # restart state: uniform over free cells
        n_free = int((occ == 0).sum())
        assert (k, j, i) == (0, 0, 2)
        assert abs(pr - 1.0 / (K * n_free)) <= 1e-6 / (K * n_free)
        b = np.full((K, H, W), 0.25, np.float32)
        b[:, occ != 0] = 0.0
        peaks = [(K - 1, H - 1, W - 1), (1, 2, 3), (1, 2, 5), (K // 2, 1, 0)]
        for q in peaks:
            b[q] = 2.0                                 # equal maxima: the lowest index wins
        loc.loc_set_belief(h, b)
        got = loc.loc_argmax(h)
        assert got[:3] == tuple(int(x) for x in np.unravel_index(np.argmax(b), b.shape))   # first of the ties
        flat = loc.loc_belief(h).reshape(-1)
        assert abs(got[3] - flat.max()) <= 1e-6 * flat.max()
    finally:
        loc.loc_destroy(h)
