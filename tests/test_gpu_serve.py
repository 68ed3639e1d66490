"""GPU tests of the serving loop (continuous batching of many sessions).

* Alone vs in the mix: a session's belief after its message stream (odometry with the 1-cell
  gate, and scans) is bit for bit the same whether the server runs it alone or among other
  sessions with their own streams, and the same as replaying the stream through loc_step and
  loc_lidar_update on a single handle with the same tile configuration.
* The plain path (one loc_step per message) gives the same result.
* Admission against the memory budget: a session that does not fit waits, its messages
  queued, and runs once another session closes.
* Latency statistics and argument checks.
"""
import math
import threading

import numpy as np
import pytest

import paper_1910_00572_gb300 as loc
from synth import floorplan, scan, trajectory, workloads

pytestmark = pytest.mark.gpu

TILE = 3
SCAN = dict(angle_min=0.0, angle_inc=math.pi / 180, r_max=6.0, beam_stride=4, sigma_r=0.1)


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1910_00572_gb300 import build
    build.build()
    loc.lib()


def session_inputs(seed, n, steps, scan_every, side=(96, 224), ks=(36, 48, 64, 72)):
    """Per session: map, parameters and a message stream [("odo", u, v, w) | ("scan", ranges)]."""
    out = []
    for i, m in enumerate(workloads.session_mix(seed, n, side=side, ks=ks)):
        occ = floorplan.office_map(m["seed"], size=m["H"], cell=m["cell"])
        walk = trajectory.random_walk(occ, m["cell"], steps, 0.05, m["seed"] + 3)
        msgs = []
        for t, (u, v, w) in enumerate(walk.odom, start=1):
            msgs.append(("odo", float(u), float(v), float(w)))
            if scan_every and t % scan_every == 0:
                z = scan.simulate_scan(occ, m["cell"], walk.poses[t], seed=m["seed"] * 31 + t, n_beams=360,
                                       r_max=SCAN["r_max"], noise_sigma=0.05, dropout=0.05, march=0.25)
                msgs.append(("scan", z))
        out.append(dict(m, occ=occ, msgs=msgs))
    return out


def params(s, storage, **kw):
    return loc.loc_params_default(H=s["H"], W=s["W"], K=s["K"], cell_m=s["cell"], storage=storage,
                                  min_shift_cells=1.0, n_samples=512, tile=TILE, **kw)


def replay_single(s, storage):
    """The same message stream through the single-session calls."""
    h = loc.loc_create(s["occ"], params(s, storage, kernel=loc.LOC_KERNEL_TILED))
    try:
        for m in s["msgs"]:
            if m[0] == "odo":
                loc.loc_step(h, *m[1:])
            else:
                loc.loc_lidar_update(h, m[1], SCAN["angle_min"], SCAN["angle_inc"], SCAN["r_max"],
                                     SCAN["beam_stride"], SCAN["sigma_r"])
        return loc.loc_belief(h), loc.loc_stats(h)
    finally:
        loc.loc_destroy(h)


def submit(srv, sid, m):
    if m[0] == "odo":
        loc.loc_server_odometry(srv, [sid], [m[1]], [m[2]], [m[3]])
    else:
        loc.loc_server_scan(srv, sid, m[1], SCAN["angle_min"], SCAN["angle_inc"], SCAN["r_max"],
                            SCAN["beam_stride"], SCAN["sigma_r"])


def serve(sessions, storage, batching=1, interleave_seed=None, budget=60e9):
    """Open every session, submit all streams (interleaved at random across sessions, each in
    its own order), drain, and read every belief back."""
    srv = loc.loc_server_create(loc.loc_server_params_default(hbm_budget_bytes=budget, storage=storage,
                                                              batching=batching, tile=TILE))
    try:
        ids = [loc.loc_server_open(srv, s["occ"], params(s, storage)) for s in sessions]
        queue = [(i, m) for i, s in enumerate(sessions) for m in s["msgs"]]
        if interleave_seed is not None:
            rng = np.random.default_rng(interleave_seed)
            pos = [0] * len(sessions)
            order = rng.permutation(np.repeat(np.arange(len(sessions)), [len(s["msgs"]) for s in sessions]))
            queue = []
            for i in order:
                queue.append((int(i), sessions[i]["msgs"][pos[i]]))
                pos[i] += 1
        for i, m in queue:
            submit(srv, ids[i], m)
        loc.loc_server_drain(srv, 120.0)
        out = []
        for sid in ids:
            state, h = loc.loc_server_session(srv, sid)
            assert state == loc.LOC_SESSION_ACTIVE
            out.append((loc.loc_belief(h), loc.loc_stats(h)))
        return out, loc.loc_server_stats(srv)
    finally:
        loc.loc_server_destroy(srv)


@pytest.mark.parametrize("storage", ["bf16", "f32"])
def test_session_is_the_same_alone_in_the_mix_and_replayed(storage):
    sess = session_inputs(21, 6, 40, 10)
    alone, st_alone = serve(sess[:1], storage)
    mixed, st_mix = serve(sess, storage, interleave_seed=5)
    single, single_stats = replay_single(sess[0], storage)
    assert np.array_equal(alone[0][0], mixed[0][0])
    assert np.array_equal(alone[0][0], single)
    assert alone[0][1]["n_propagations"] == single_stats["n_propagations"] > 5
    assert alone[0][1]["logscale"] == single_stats["logscale"]
    # the other sessions of the mix are each their own replay too
    for s, (b, _) in zip(sess[1:3], mixed[1:3]):
        assert np.array_equal(b, replay_single(s, storage)[0])
    assert st_mix["n_scans"] == sum(1 for s in sess for m in s["msgs"] if m[0] == "scan")
    assert st_mix["n_messages"] == sum(len(s["msgs"]) for s in sess)
    assert st_mix["n_propagations"] == sum(r[1]["n_propagations"] for r in mixed)
    assert st_mix["mean_batch"] >= 1.0
    assert 0 < st_mix["step_p50_ms"] <= st_mix["step_p99_ms"] <= st_mix["step_max_ms"]
    assert 0 < st_mix["scan_p50_ms"] <= st_mix["scan_p99_ms"]


def test_plain_path_gives_the_same_beliefs():
    sess = session_inputs(23, 3, 30, 15)
    plain, st = serve(sess, "f32", batching=0, interleave_seed=1)
    batched, _ = serve(sess, "f32", batching=1, interleave_seed=2)
    for (a, _), (b, _) in zip(plain, batched):
        assert np.array_equal(a, b)
    assert st["mean_batch"] == 0.0 and st["n_propagations"] > 0


def test_admission_waits_for_memory_and_runs_after_a_close():
    sess = session_inputs(25, 3, 20, 0, side=(128, 129), ks=(36,))
    need = [loc.loc_session_bytes(params(s, "bf16")) for s in sess]
    budget = need[0] + need[1] + need[2] // 2            # room for two of the three
    srv = loc.loc_server_create(loc.loc_server_params_default(hbm_budget_bytes=budget, storage="bf16", tile=TILE))
    try:
        ids = [loc.loc_server_open(srv, s["occ"], params(s, "bf16")) for s in sess]
        for i, s in enumerate(sess):
            for m in s["msgs"]:
                submit(srv, ids[i], m)
        loc.loc_server_drain(srv, 60.0)
        st = loc.loc_server_stats(srv)
        assert (st["n_active"], st["n_pending"]) == (2, 1)
        assert st["bytes_used"] == need[0] + need[1] <= budget
        assert loc.loc_server_session(srv, ids[2])[0] == loc.LOC_SESSION_PENDING
        loc.loc_server_close(srv, ids[0])
        loc.loc_server_drain(srv, 60.0)
        for _ in range(200):                                  # the close and admission happen on the worker
            if loc.loc_server_session(srv, ids[2])[0] == loc.LOC_SESSION_ACTIVE:
                break
            threading.Event().wait(0.01)
        loc.loc_server_drain(srv, 60.0)
        state, h = loc.loc_server_session(srv, ids[2])
        assert state == loc.LOC_SESSION_ACTIVE
        assert loc.loc_server_session(srv, ids[0])[0] == loc.LOC_SESSION_CLOSED
        assert np.array_equal(loc.loc_belief(h), replay_single(sess[2], "bf16")[0])
    finally:
        loc.loc_server_destroy(srv)


def test_server_rejects_bad_requests():
    sess = session_inputs(27, 1, 2, 0, side=(96, 97), ks=(36,))
    s = sess[0]
    srv = loc.loc_server_create(loc.loc_server_params_default(hbm_budget_bytes=1e9, storage="f32", tile=TILE))
    try:
        with pytest.raises(loc.LocError) as e:
            loc.loc_server_open(srv, s["occ"], params(s, "f32", kernel=loc.LOC_KERNEL_GENERIC))
        assert e.value.status == loc.LOC_ERR_INVALID_ARG
        big = dict(s, H=4096, W=4096, occ=np.zeros((4096, 4096), np.uint8))
        with pytest.raises(loc.LocError):
            loc.loc_server_open(srv, big["occ"], params(big, "f32"))       # never fits 1 GB
        sid = loc.loc_server_open(srv, s["occ"], params(s, "f32"))
        with pytest.raises(loc.LocError):
            loc.loc_server_odometry(srv, [sid + 1], [0.1], [0.0], [0.0])
        with pytest.raises(loc.LocError):
            loc.loc_server_odometry(srv, [sid], [math.nan], [0.0], [0.0])
        loc.loc_server_drain(srv, 30.0)
        assert loc.loc_server_stats(srv)["n_active"] == 1
    finally:
        loc.loc_server_destroy(srv)


@pytest.mark.slow
def test_serve256_sessions_one_served_tick_sampled_against_oracle():
    """Sessions of the served workload at full size -- the largest (1984 x 1984 x 72, 283 M states),
    a mid-sized and the smallest -- served together in BF16 the way the benchmark serves them
    (batched launch, autotuned tile, the 1-cell gate), one odometry message each.  From a belief
    with sharp peaks set through the session handle, sampled states of each session's propagated
    tensor are recomputed one by one from the definitions by the oracle (Alg. 1's propagation
    from the same stored input): each within one BF16 rounding step of its own exact value
    plus the FP32 error (tests/bounds.py), and the tensor sums to 1."""
    import bounds
    from oracle import filter as F
    from oracle.odometry import Odometry
    from synth import fields
    wl = workloads.get("serve256")
    mix = workloads.make_sessions(wl, 2)
    order = sorted(range(len(mix)), key=lambda q: -mix[q]["H"] * mix[q]["W"] * mix[q]["K"])
    picks = [mix[order[0]], mix[order[len(order) // 2]], mix[order[-1]]]
    u, v, w = 0.043, -0.029, 0.004                    # 1.04 cells: opens the 1-cell gate
    srv = loc.loc_server_create(loc.loc_server_params_default(hbm_budget_bytes=wl["hbm_budget_gb"] * 1e9,
                                                              storage="bf16", batching=1, tile=0))
    try:
        ids = [loc.loc_server_open(srv, s["occ"], loc.loc_params_default(
            H=s["H"], W=s["W"], K=s["K"], cell_m=s["cell"], storage="bf16",
            min_shift_cells=wl["min_shift_cells"], n_samples=wl["n_samples"])) for s in picks]
        loc.loc_server_drain(srv, 300.0)
        befores = []
        for q, (s, sid) in enumerate(zip(picks, ids)):
            state, h = loc.loc_server_session(srv, sid)
            assert state == loc.LOC_SESSION_ACTIVE
            loc.loc_set_belief(h, fields.belief_like(s["occ"], s["K"], seed=31 + q, dtype=np.float32))
            befores.append(loc.loc_belief(h))          # the stored BF16 input, normalised
        loc.loc_server_odometry(srv, ids, [u] * len(ids), [v] * len(ids), [w] * len(ids))
        loc.loc_server_drain(srv, 300.0)
        assert loc.loc_server_stats(srv)["n_propagations"] == len(ids)
        rng = np.random.default_rng(12)
        for s, sid, before in zip(picks, ids, befores):
            _, h = loc.loc_server_session(srv, sid)
            got = loc.loc_belief(h)
            Z = loc.loc_stats(h)["last_Z"]
            K, H, W = s["K"], s["H"], s["W"]
            odo = Odometry(K, s["cell"])
            odo.add(u, v, w)
            M = F.traversability(s["occ"])
            g = F.motion_kernel(wl["sigma_xy_cells"], wl["sigma_theta_bins"])
            idx = [(int(rng.integers(K)), int(rng.integers(H)), int(rng.integers(W))) for _ in range(1500)]
            for qq in np.argpartition(before.reshape(-1), -4)[-4:]:
                k, rem = divmod(int(qq), H * W)
                j, i = rem // W, rem % W
                idx += [(k, jj, ii) for jj in range(max(0, j - 2), min(H, j + 3))
                        for ii in range(max(0, i - 2), min(W, i + 3))]
            T = F.propagate_at(before.astype(np.float64), M, odo.shifts(), g, idx)
            gotT = np.array([got[k, j, i] for (k, j, i) in idx], np.float64) * Z
            bad = np.flatnonzero(np.abs(gotT - T) > bounds.bf16_step_bound(T))
            assert bad.size == 0, (H, K, [(idx[b], gotT[b], T[b]) for b in bad[:5]])
            assert abs(got.astype(np.float64).sum() - 1.0) < 1e-4
    finally:
        loc.loc_server_destroy(srv)
