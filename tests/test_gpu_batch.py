"""GPU tests of the batched propagation (one persistent launch over many sessions).

* A session's result must not depend on the batch it is in: with the same tile configuration,
  a session stepped in a batch is compared bit for bit with the same session stepped alone by
  loc_step, in FP32 and BF16, for a batch of one and for mixes of uneven H x W x K, with and
  without the CUDA graph.
* FP32 batches are compared with the FP64 oracle within 1e-6 absolute (and 2e-5 of the largest
  value) of the normalised belief.
* The per-session gate, the autotuner's dry run (which must leave every session unchanged),
  interleaving batch ticks with single-session steps, and argument checks.
"""
import numpy as np
import pytest

import bounds
import paper_1910_00572_gb300 as loc
from oracle import filter as F
from synth import fields, floorplan, trajectory, workloads

pytestmark = pytest.mark.gpu

ABS_TOL = 1e-6
REL_TOL = 2e-5


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1910_00572_gb300 import build
    build.build()
    loc.lib()


def mix_inputs(seed, n, steps, side=(96, 320), ks=(36, 48, 64, 72), dt=0.05):
    """Maps, odometry and initial beliefs of n sessions of uneven size (office plans)."""
    out = []
    for m in workloads.session_mix(seed, n, side=side, ks=ks):
        occ = floorplan.office_map(m["seed"], size=m["H"], cell=m["cell"])
        walk = trajectory.random_walk(occ, m["cell"], steps, dt, m["seed"] + 17)
        out.append(dict(m, occ=occ, odom=np.asarray(walk.odom, np.float64)))
    return out


def create(s, storage="f32", tile=0, **kw):
    p = loc.loc_params_default(H=s["H"], W=s["W"], K=s["K"], cell_m=s["cell"], storage=storage,
                               kernel=loc.LOC_KERNEL_TILED, tile=tile, **kw)
    return loc.loc_create(s["occ"], p)


def run_batch(sess, storage, tile, use_graph, steps, set_beliefs=None):
    hs = [create(s, storage) for s in sess]
    try:
        if set_beliefs is not None:
            for h, b in zip(hs, set_beliefs):
                loc.loc_set_belief(h, b)
        b = loc.loc_batch_create(hs, tile=tile, use_graph=use_graph)
        try:
            info = loc.loc_batch_info(b)
            for t in range(steps):
                odo = np.stack([s["odom"][t] for s in sess])
                loc.loc_batch_step(b, odo[:, 0], odo[:, 1], odo[:, 2])
            loc.loc_batch_sync(b)
        finally:
            loc.loc_batch_destroy(b)
        return [loc.loc_belief(h) for h in hs], [loc.loc_stats(h) for h in hs], info
    finally:
        for h in hs:
            loc.loc_destroy(h)


def run_alone(s, storage, tile, steps, belief=None):
    h = create(s, storage, tile=tile)
    try:
        if belief is not None:
            loc.loc_set_belief(h, belief)
        for t in range(steps):
            loc.loc_step(h, *s["odom"][t])
        return loc.loc_belief(h), loc.loc_stats(h)
    finally:
        loc.loc_destroy(h)


@pytest.mark.parametrize("storage", ["f32", "bf16"])
@pytest.mark.parametrize("tile", [1, 2, 3])
def test_batch_of_one_is_bitwise_the_single_session(storage, tile):
    sess = mix_inputs(5, 1, 12, side=(150, 260))
    got, st, info = run_batch(sess, storage, tile, True, 12)
    assert info["tile"] == tile and info["grid"] > 0
    want, wst = run_alone(sess[0], storage, tile, 12)
    assert np.array_equal(got[0], want)
    assert st[0]["logscale"] == wst["logscale"] and st[0]["n_propagations"] == 12


@pytest.mark.parametrize("storage,use_graph", [("f32", True), ("bf16", True), ("f32", False), ("f16", True)])
def test_mixed_batch_equals_each_session_alone(storage, use_graph):
    sess = mix_inputs(3, 6, 10)
    beliefs = [fields.belief_like(s["occ"], s["K"], seed=s["seed"], dtype=np.float32) for s in sess]
    got, st, info = run_batch(sess, storage, 0, use_graph, 10, set_beliefs=beliefs)
    assert 1 <= info["tile"] <= loc.LOC_BATCH_CONFIGS
    for s, b, g, gs in zip(sess, beliefs, got, st):
        want, ws = run_alone(s, storage, info["tile"], 10, belief=b)
        assert np.array_equal(g, want), (s["H"], s["K"])
        assert gs["logscale"] == ws["logscale"]


def test_fp32_batch_matches_oracle():
    rng = np.random.default_rng(4)
    shapes = [(64, 64, 16, 0.1), (72, 96, 9, 0.05), (40, 64, 36, 0.05), (33, 8, 8, 0.05)]
    sess = []
    for H, W, K, cell in shapes:
        occ = (rng.random((H, W)) < 0.15).astype(np.uint8)
        occ[H // 2, W // 2] = 0
        odom = np.column_stack([rng.uniform(-2, 2, 12) * cell, rng.uniform(-2, 2, 12) * cell,
                                rng.uniform(-0.3, 0.3, 12)])
        sess.append(dict(H=H, W=W, K=K, cell=cell, occ=occ, odom=odom))
    beliefs = [fields.belief_like(s["occ"], s["K"], seed=s["K"], dtype=np.float32) for s in sess]
    got, _, _ = run_batch(sess, "f32", 0, True, 12, set_beliefs=beliefs)
    for s, b, g in zip(sess, beliefs, got):
        ref = F.Filter(s["occ"], s["K"], s["cell"])
        ref.B = b.astype(np.float64) / b.astype(np.float64).sum()
        for t in range(12):
            ref.step(*s["odom"][t])
        err = np.abs(g.astype(np.float64) - ref.B).max()
        assert err <= ABS_TOL and err <= REL_TOL * ref.B.max(), (s["H"], s["W"], s["K"], err)


def test_gate_moves_only_sessions_past_the_threshold():
    sess = mix_inputs(7, 4, 30, side=(96, 200))
    hs = [create(s, "f32", tile=3, min_shift_cells=1.0) for s in sess]
    alone = [create(s, "f32", tile=3, min_shift_cells=1.0) for s in sess]
    b = loc.loc_batch_create(hs, tile=3)
    try:
        scale = np.array([1.0, 0.05, 1.0, 0.1])
        for t in range(30):
            # sessions 0 and 2 move every tick; 1 and 3 creep and pass the 1-cell gate rarely
            odo = np.stack([s["odom"][t] for s in sess]) * scale[:, None]
            expect = sum(loc.loc_step(a, *o) == loc.LOC_OK for a, o in zip(alone, odo))
            moved = loc.loc_batch_step(b, odo[:, 0], odo[:, 1], odo[:, 2])
            assert moved == expect, t
        loc.loc_batch_sync(b)
        for h, a in zip(hs, alone):
            assert np.array_equal(loc.loc_belief(h), loc.loc_belief(a))
            assert loc.loc_stats(h)["n_propagations"] == loc.loc_stats(a)["n_propagations"]
    finally:
        loc.loc_batch_destroy(b)
        for h in hs + alone:
            loc.loc_destroy(h)


def test_autotune_dry_run_leaves_sessions_unchanged():
    sess = mix_inputs(9, 3, 1)
    hs = [create(s, "bf16") for s in sess]
    try:
        for h, s in zip(hs, sess):
            loc.loc_set_belief(h, fields.belief_like(s["occ"], s["K"], seed=3, dtype=np.float32))
        before = [loc.loc_belief(h) for h in hs]
        stats = [loc.loc_stats(h) for h in hs]
        b = loc.loc_batch_create(hs, tile=0, use_graph=True)
        try:
            info = loc.loc_batch_info(b)
        finally:
            loc.loc_batch_destroy(b)
        assert 1 <= info["tile"] <= loc.LOC_BATCH_CONFIGS
        assert all(ms > 0 for ms in info["tune_ms"])
        assert info["tune_ms"][info["tile"] - 1] == min(info["tune_ms"])
        for h, x, s0 in zip(hs, before, stats):
            assert np.array_equal(loc.loc_belief(h), x)
            s1 = loc.loc_stats(h)
            assert s1["logscale"] == s0["logscale"] and s1["n_propagations"] == 0
    finally:
        for h in hs:
            loc.loc_destroy(h)


def test_batch_ticks_interleave_with_single_steps():
    sess = mix_inputs(11, 3, 16, side=(96, 200))
    hs = [create(s, "f32", tile=2) for s in sess]
    b = loc.loc_batch_create(hs, tile=2)
    try:
        for t in range(16):
            if t % 3 == 1:
                for h, s in zip(hs, sess):
                    loc.loc_step(h, *s["odom"][t])
            else:
                odo = np.stack([s["odom"][t] for s in sess])
                loc.loc_batch_step(b, odo[:, 0], odo[:, 1], odo[:, 2])
        loc.loc_batch_sync(b)
        for h, s in zip(hs, sess):
            want, _ = run_alone(s, "f32", 2, 16)
            assert np.array_equal(loc.loc_belief(h), want)
    finally:
        loc.loc_batch_destroy(b)
        for h in hs:
            loc.loc_destroy(h)


def test_batch_rejects_bad_groups():
    sess = mix_inputs(13, 2, 1, side=(96, 128))
    a = create(sess[0], "f32")
    c = create(sess[1], "bf16")
    p = loc.loc_params_default(H=sess[1]["H"], W=sess[1]["W"], K=sess[1]["K"], cell_m=0.05,
                               kernel=loc.LOC_KERNEL_GENERIC)
    g = loc.loc_create(sess[1]["occ"], p)
    try:
        for group in ([a, a], [a, c], [a, g]):
            with pytest.raises(loc.LocError) as e:
                loc.loc_batch_create(group)
            assert e.value.status == loc.LOC_ERR_INVALID_ARG
        with pytest.raises(loc.LocError):
            loc.loc_batch_create([a], tile=loc.LOC_BATCH_CONFIGS + 1)
        b = loc.loc_batch_create([a], tile=1)
        try:
            with pytest.raises(loc.LocError) as e:
                loc.loc_batch_step(b, [np.nan], [0.0], [0.0])
            assert e.value.status == loc.LOC_ERR_INVALID_ARG
            assert loc.loc_stats(a)["n_propagations"] == 0
        finally:
            loc.loc_batch_destroy(b)
    finally:
        for h in (a, c, g):
            loc.loc_destroy(h)


@pytest.mark.slow
@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_batch64_full_size_sampled_against_oracle(storage):
    """The 64-session workload at full size (0.95 G cells), one batched tick in the launch
    configuration the benchmark times (autotuned tile, CUDA graph): on four sessions (the two
    largest and two smaller, different K), sampled states are recomputed one by one from the
    definitions by the oracle from the same input belief.  FP32: 1e-6; BF16: each state within
    one BF16 rounding step of its own exact value plus the FP32 error, and the argmax
    state as large as every checked state."""
    from oracle.odometry import Odometry
    wl = workloads.get("batch64")
    sess = workloads.make_sessions(wl, 2)
    order = sorted(range(len(sess)), key=lambda q: -sess[q]["H"] * sess[q]["W"] * sess[q]["K"])
    check = [order[0], order[1], order[len(order) // 2], order[-1]]
    hs = [loc.loc_create(s["occ"], loc.loc_params_default(H=s["H"], W=s["W"], K=s["K"], cell_m=s["cell"],
                                                          storage=storage)) for s in sess]
    try:
        for q in check:
            loc.loc_set_belief(hs[q], fields.belief_like(sess[q]["occ"], sess[q]["K"], seed=q, dtype=np.float32))
        before = {q: loc.loc_belief(hs[q]).astype(np.float64) for q in check}
        b = loc.loc_batch_create(hs, tile=0, use_graph=True)
        try:
            odo = np.stack([s["odom"][0] for s in sess])
            assert loc.loc_batch_step(b, odo[:, 0], odo[:, 1], odo[:, 2]) == len(sess)
            loc.loc_batch_sync(b)
        finally:
            loc.loc_batch_destroy(b)
        for q in check:
            s = sess[q]
            K, H, W = s["K"], s["H"], s["W"]
            got = loc.loc_belief(hs[q]).astype(np.float64)
            Z = loc.loc_stats(hs[q])["last_Z"]
            od = Odometry(K, s["cell"])
            od.add(*s["odom"][0])
            g = F.motion_kernel(wl["sigma_xy_cells"], wl["sigma_theta_bins"])
            rng = np.random.default_rng(q)
            idx = [(int(rng.integers(K)), int(rng.integers(H)), int(rng.integers(W))) for _ in range(400)]
            for flat in np.argsort(before[q].reshape(-1))[-10:]:
                k, rem = divmod(int(flat), H * W)
                idx.append((k, rem // W, rem % W))
            T = F.propagate_at(before[q], F.traversability(s["occ"]), od.shifts(), g, idx)
            gotT = np.array([got[k, j, i] for (k, j, i) in idx]) * Z
            err = np.abs(gotT - T).max()
            if storage == "f32":
                assert err <= ABS_TOL and err <= REL_TOL * before[q].max(), (q, err)
            else:
                # per element: one BF16 rounding step of that state's own value plus
                # the FP32 propagation error (tests/bounds.py)
                bound = bounds.bf16_step_bound(T)
                bad = np.flatnonzero(np.abs(gotT - T) > bound)
                assert bad.size == 0, (q, [(idx[b], gotT[b], T[b], bound[b]) for b in bad[:5]])
                # the batch's argmax state (fused or by the pass) holds at least every checked
                # state's exact value, to within the rounding of both
                ak, aj, ai, _ = loc.loc_argmax(hs[q])
                Ta = F.propagate_at(before[q], F.traversability(s["occ"]), od.shifts(), g, [(ak, aj, ai)])[0]
                assert Ta >= T.max() - 2.0 * bounds.bf16_step_bound(T.max()), (q, Ta, T.max())
            assert abs(got.sum() - 1.0) < 1e-4
    finally:
        for h in hs:
            loc.loc_destroy(h)
