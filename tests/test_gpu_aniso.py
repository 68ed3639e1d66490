"""GPU parity of the propagation with anisotropic motion noise (Eq. 5-6, sigma_x != sigma_y)
through the C-ABI against the FP64 oracle ``oracle.aniso``.

The bar is the isotropic path's: FP32 storage agrees to 1e-6 absolute and 2e-5 of the tensor's
maximum (one step rounds the bilinear taps, the theta sum, an x/y stencil of up to 81 taps and
its map sum, each term a relative 2^-24; the stencil is evaluated in FP32 from the channel's
heading and its rounding largely cancels in T_k / G_k, which is a weighted mean with the same
weights); reduced precision keeps L1 <= 1e-2 and the same argmax.  A nearly isotropic session
on this path also matches the isotropic oracle, which pins the kernel to a second oracle.
"""
import math

import numpy as np
import pytest

import paper_1910_00572_gb300 as loc
from oracle import aniso as A
from oracle import filter as F
from oracle import readout as R
from synth import fields, floorplan, trajectory

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


def check_close(gpu, ref):
    err = np.abs(gpu.astype(np.float64) - ref)
    assert err.max() <= ABS_TOL, err.max()
    assert err.max() <= REL_TOL * ref.max(), (err.max(), ref.max())
    return float(err.max())


@pytest.mark.parametrize("H,W", [(52, 75), (56, 72)], ids=["plain loads", "TMA boxes"])
def test_trajectory_matches_oracle(H, W):
    """A walk with turns on a crop of a rooms map that leaves a ragged tail of the 32 x 32
    tiles in both directions, radius 4 in x/y and 3 in theta, from a peaked belief.  A row
    pitch of 75 cells takes the plain-load input path, 72 the TMA path."""
    occ = floorplan.rooms_map(4, size=80)[:H, :W].copy()
    K, cell, sx, sy, sth = 16, 0.1, 1.2, 0.5, 1.0
    walk = trajectory.random_walk(occ, cell, 12, 0.1, 7)
    b0 = fields.belief_like(occ, K, seed=3, dtype=np.float32)
    h = make(occ, K, cell, sigma_xy_cells=sx, sigma_cross_cells=sy, sigma_theta_bins=sth)
    ref = A.Filter(occ, K, cell, sx, sy, sth)
    ref.B = b0.astype(np.float64) / b0.astype(np.float64).sum()
    worst = 0.0
    try:
        loc.loc_set_belief(h, b0)
        for t, (u, v, w) in enumerate(walk.odom, start=1):
            loc.loc_step(h, u, v, w)
            ref.step(u, v, w)
            worst = max(worst, check_close(loc.loc_belief(h), ref.B))
            st = loc.loc_stats(h)
            assert abs(st["last_Z"] - ref.last_Z) <= 1e-6 * ref.last_Z, t
            assert abs(st["logscale"] - ref.logscale) <= 1e-5 * max(1.0, abs(ref.logscale)), t
            assert st["n_propagations"] == t
            assert abs(st["theta"] - ref.odo.theta) <= 1e-12
        assert (loc.loc_belief(h)[:, occ != 0] == 0.0).all()
    finally:
        loc.loc_destroy(h)
    print(f"worst abs error {worst:.3e}")


CASES = [
    # H, W, K, sigma along, sigma across, sigma theta, r_xy, motion (cells, cells, rad), label
    (40, 70, 8, 1.2, 0.5, 1.0, -1, (0.6, -0.3, 0.7), "long along the heading"),
    (37, 45, 12, 0.4, 1.1, 0.8, -1, (-0.4, 0.9, -1.9), "wide across the heading"),
    (1, 90, 4, 1.0, 0.5, 1.0, -1, (2.2, 0.0, 0.3), "single row"),
    (70, 1, 4, 1.0, 0.5, 1.0, -1, (0.0, 1.6, 0.0), "single column"),
    (33, 33, 1, 1.0, 0.6, 1.0, -1, (0.25, 0.75, 2.0), "one bin"),
    (30, 50, 3, 0.9, 0.4, 1.3, -1, (0.5, 0.2, 0.4), "K < theta kernel"),
    (48, 48, 16, 1.3, 0.6, 0.0, 2, (-0.6, 0.35, -0.2), "truncated radius, no theta blur"),
    (40, 40, 6, 1.0, 0.5, 1.0, -1, (25.3, -14.6, 0.0), "shift beyond the tile"),
    (35, 66, 10, 0.8, 1.3, 1.0, -1, (0.0, 0.0, -7.4), "heading wraps below zero"),
]


@pytest.mark.parametrize("H,W,K,sx,sy,sth,rxy,mot,label", CASES, ids=[c[-1] for c in CASES])
def test_edge_cases_match_oracle(H, W, K, sx, sy, sth, rxy, mot, label):
    rng = np.random.default_rng(H * 1000 + W)
    occ = (rng.random((H, W)) < 0.15).astype(np.uint8)
    occ[H // 2, W // 2] = 0
    cell = 0.1
    b = fields.belief_like(occ, K, seed=H + W, dtype=np.float32)
    h = make(occ, K, cell, sigma_xy_cells=sx, sigma_cross_cells=sy, sigma_theta_bins=sth, r_xy=rxy)
    ref = A.Filter(occ, K, cell, sx, sy, sth, r_xy=None if rxy < 0 else rxy)
    ref.B = b.astype(np.float64) / b.astype(np.float64).sum()
    try:
        loc.loc_set_belief(h, b)
        for _ in range(3):
            u, v, w = mot[0] * cell, mot[1] * cell, mot[2]
            loc.loc_step(h, u, v, w)
            ref.step(u, v, w)
            if ref.last_Z == 0.0:
                break
            check_close(loc.loc_belief(h), ref.B)
    finally:
        loc.loc_destroy(h)


def test_equal_sigmas_take_the_isotropic_path():
    """sigma_cross == sigma_xy is the isotropic session, bit for bit."""
    occ = floorplan.rooms_map(5, size=64)
    walk = trajectory.random_walk(occ, 0.1, 6, 0.1, 2)
    out = []
    for cross in (0.0, 0.5):
        h = make(occ, 8, 0.1, sigma_xy_cells=0.5, sigma_cross_cells=cross, kernel=loc.LOC_KERNEL_GENERIC)
        try:
            for u, v, w in walk.odom:
                loc.loc_step(h, u, v, w)
            out.append(loc.loc_belief(h))
        finally:
            loc.loc_destroy(h)
    assert np.array_equal(out[0], out[1])


def test_nearly_isotropic_session_matches_the_isotropic_oracle():
    """sigma_x and sigma_y a relative 1e-9 apart run the anisotropic kernel, whose result is then
    the separable filter of Eq. 5 with a single sigma (``oracle.filter``) to FP32 accuracy."""
    occ = floorplan.rooms_map(6, size=72)[:61, :70].copy()
    K, cell = 12, 0.1
    walk = trajectory.random_walk(occ, cell, 8, 0.1, 9)
    b0 = fields.belief_like(occ, K, seed=5, dtype=np.float32)
    h = make(occ, K, cell, sigma_xy_cells=0.7, sigma_cross_cells=0.7 * (1 + 1e-9), sigma_theta_bins=1.1)
    ref = F.Filter(occ, K, cell, 0.7, 1.1)
    ref.B = b0.astype(np.float64) / b0.astype(np.float64).sum()
    try:
        loc.loc_set_belief(h, b0)
        for u, v, w in walk.odom:
            loc.loc_step(h, u, v, w)
            ref.step(u, v, w)
            check_close(loc.loc_belief(h), ref.B)
    finally:
        loc.loc_destroy(h)


def test_all_mass_removed_restarts_and_steps_on():
    """Every hypothesis walks into a wall: Z = 0, the belief restarts uniform over the free
    cells, and the next step propagates that restart state (the kernel's reinit input)."""
    occ = np.ones((30, 40), np.uint8)
    occ[8:22, 10:30] = 0
    h = make(occ, 4, 1.0, sigma_xy_cells=0.3, sigma_cross_cells=0.2, sigma_theta_bins=0.0, r_xy=1)
    ref = A.Filter(occ, 4, 1.0, 0.3, 0.2, 0.0, r_xy=1)
    b = np.zeros((4, 30, 40), np.float32)
    b[:, 14, 12] = 0.25                                  # mass two cells from the left wall
    ref.B = b.astype(np.float64)
    try:
        loc.loc_set_belief(h, b)
        loc.loc_step(h, 25.0, 0.0, 0.0)                  # 25 cells: out of the room in every bin
        ref.step(25.0, 0.0, 0.0)
        st = loc.loc_stats(h)
        assert st["n_reinit"] == 1 and st["last_Z"] == 0.0 and ref.last_Z == 0.0
        M = (occ == 0).astype(np.float64)
        assert np.abs(loc.loc_belief(h) - F.uniform_belief(M, 4)).max() <= 1e-9
        loc.loc_step(h, 1.5, -0.5, 0.4)
        ref.step(1.5, -0.5, 0.4)
        check_close(loc.loc_belief(h), ref.B)
        assert loc.loc_stats(h)["n_reinit"] == 1
    finally:
        loc.loc_destroy(h)


@pytest.mark.parametrize("storage", ["bf16", "f16"])
def test_reduced_precision_trajectory_l1_and_argmax(storage):
    occ = floorplan.rooms_map(7, size=64)
    K, cell = 16, 0.1
    walk = trajectory.random_walk(occ, cell, 30, 0.1, 11)
    h = make(occ, K, cell, storage=storage, sigma_xy_cells=1.0, sigma_cross_cells=0.5)
    ref = A.Filter(occ, K, cell, 1.0, 0.5, 1.0)
    b0 = fields.belief_like(occ, K, seed=8, dtype=np.float32)
    ref.B = b0.astype(np.float64) / b0.astype(np.float64).sum()
    worst = 0.0
    try:
        loc.loc_set_belief(h, b0)
        for t, (u, v, w) in enumerate(walk.odom, start=1):
            loc.loc_step(h, u, v, w)
            ref.step(u, v, w)
            if t % 5 == 0:
                b = loc.loc_belief(h).astype(np.float64)
                l1 = np.abs(b - ref.B).sum()
                worst = max(worst, l1)
                assert l1 <= 1e-2, (t, l1)
                k, j, i, _ = R.argmax_pose(ref.B)
                top2 = np.sort(ref.B.reshape(-1))[-2:]
                if top2[1] - top2[0] > 2 * 1e-2 * top2[1]:
                    assert loc.loc_argmax(h)[:3] == (k, j, i), t
    finally:
        loc.loc_destroy(h)
    print(f"{storage}: worst L1 {worst:.3e}")


def test_batching_refuses_and_the_plain_server_path_runs_anisotropic_sessions():
    occ = floorplan.rooms_map(8, size=64)
    prm = dict(H=64, W=64, K=8, cell_m=0.1, sigma_xy_cells=1.0, sigma_cross_cells=0.4)
    h = loc.loc_create(occ, loc.loc_params_default(**prm))
    try:
        with pytest.raises(loc.LocError) as e:
            loc.loc_batch_create([h])
        assert e.value.status == loc.LOC_ERR_INVALID_ARG
    finally:
        loc.loc_destroy(h)
    walk = trajectory.random_walk(occ, 0.1, 10, 0.1, 4)
    srv = loc.loc_server_create(loc.loc_server_params_default(hbm_budget_bytes=1e9, storage="f32", batching=1))
    try:
        with pytest.raises(loc.LocError):
            loc.loc_server_open(srv, occ, loc.loc_params_default(**prm))
    finally:
        loc.loc_server_destroy(srv)
    srv = loc.loc_server_create(loc.loc_server_params_default(hbm_budget_bytes=1e9, storage="f32", batching=0))
    try:
        sid = loc.loc_server_open(srv, occ, loc.loc_params_default(**prm))
        for u, v, w in walk.odom:
            loc.loc_server_odometry(srv, [sid], [u], [v], [w])
        loc.loc_server_drain(srv, 60.0)
        state, hs = loc.loc_server_session(srv, sid)
        assert state == loc.LOC_SESSION_ACTIVE
        got = loc.loc_belief(hs)
    finally:
        loc.loc_server_destroy(srv)
    h = loc.loc_create(occ, loc.loc_params_default(**prm))
    try:
        for u, v, w in walk.odom:
            loc.loc_step(h, u, v, w)
        assert np.array_equal(got, loc.loc_belief(h))
    finally:
        loc.loc_destroy(h)
