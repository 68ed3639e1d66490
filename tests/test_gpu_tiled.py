"""GPU parity of the TMA-tiled propagation kernel (x/y radius 2, theta radius 3) against the
FP64 oracle and against the generic kernel, on shapes that stress its tiling: ragged tile
edges, widths that are not a multiple of the 64-cell tile, K not a multiple of the 7-deep
theta ring, the smallest K it accepts, shifts larger than a tile, the uniform-restart input,
and reduced-precision storage."""
import numpy as np
import pytest

import paper_1910_00572_gb300 as loc
from oracle import filter as F
from oracle import readout as R
from synth import fields, floorplan, workloads

pytestmark = pytest.mark.gpu

ABS_TOL = 1e-6
REL_TOL = 2e-5


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1910_00572_gb300 import build
    build.build()
    loc.lib()


def make(occ, K, cell, kernel=loc.LOC_KERNEL_TILED, **kw):
    p = loc.loc_params_default(H=occ.shape[0], W=occ.shape[1], K=K, cell_m=cell, kernel=kernel, **kw)
    return loc.loc_create(occ, p)


def close(gpu, ref, abs_tol=ABS_TOL, rel_tol=REL_TOL):
    err = np.abs(gpu.astype(np.float64) - ref).max()
    assert err <= abs_tol and err <= rel_tol * ref.max(), (err, ref.max())


SHAPES = [
    # (H, W, K, motion per step in cells (u, v) and w)
    (64, 64, 16, (0.3, -0.7, 0.05)),
    (70, 136, 9, (1.7, 0.4, -0.1)),
    (33, 8, 8, (0.5, 0.25, 0.0)),
    (100, 200, 13, (-2.6, 1.1, 0.2)),
    (41, 72, 72, (0.9, 0.9, 0.03)),
    (48, 96, 10, (37.5, -20.25, 0.0)),
]


@pytest.mark.parametrize("tile", list(range(1, 19)))
@pytest.mark.parametrize("H,W,K,mot", SHAPES, ids=[f"{s[0]}x{s[1]}x{s[2]}" for s in SHAPES])
def test_tiled_matches_oracle_and_generic(H, W, K, mot, tile):
    rng = np.random.default_rng(H * 7 + W * 3 + K)
    occ = (rng.random((H, W)) < 0.2).astype(np.uint8)
    occ[H // 2, W // 2] = 0
    cell = 0.05
    b = fields.belief_like(occ, K, seed=K, dtype=np.float32)
    ht = make(occ, K, cell, tile=tile)
    hg = make(occ, K, cell, kernel=loc.LOC_KERNEL_GENERIC)
    ref = F.Filter(occ, K, cell)
    ref.B = b.astype(np.float64) / b.astype(np.float64).sum()
    try:
        loc.loc_set_belief(ht, b)
        loc.loc_set_belief(hg, b)
        for _ in range(3):
            u, v, w = mot[0] * cell, mot[1] * cell, mot[2]
            for h in (ht, hg):
                loc.loc_step(h, u, v, w)
            ref.step(u, v, w)
            if ref.last_Z == 0.0:
                break
            bt, bg = loc.loc_belief(ht), loc.loc_belief(hg)
            close(bt, ref.B)
            close(bt, bg.astype(np.float64))
            assert abs(loc.loc_stats(ht)["last_Z"] - ref.last_Z) <= 1e-6 * max(ref.last_Z, 1e-30)
    finally:
        loc.loc_destroy(ht)
        loc.loc_destroy(hg)


@pytest.mark.parametrize("tile", [1, 3, 6, 8, 13, 14, 15, 16, 17])
def test_largest_theta_count(tile):
    """K = LOC_MAX_K (256 bins): the theta ring and the wrap planes at the largest size."""
    H, W, K = 20, 72, 256
    rng = np.random.default_rng(256)
    occ = (rng.random((H, W)) < 0.1).astype(np.uint8)
    b = fields.belief_like(occ, K, seed=3, dtype=np.float32)
    h = make(occ, K, 0.05, tile=tile)
    ref = F.Filter(occ, K, 0.05)
    ref.B = b.astype(np.float64) / b.astype(np.float64).sum()
    try:
        loc.loc_set_belief(h, b)
        for u, v, w in [(0.031, -0.012, 0.07), (-0.02, 0.044, -0.03)]:
            loc.loc_step(h, u, v, w)
            ref.step(u, v, w)
            close(loc.loc_belief(h), ref.B)
    finally:
        loc.loc_destroy(h)


def test_tiled_first_step_reads_uniform_and_walls_hold_no_mass():
    occ = floorplan.rooms_map(9, size=64)
    h = make(occ, 16, 0.1)
    ref = F.Filter(occ, 16, 0.1)
    try:
        for (u, v, w) in [(0.04, 0.01, 0.1), (0.02, -0.05, -0.2)]:
            loc.loc_step(h, u, v, w)
            ref.step(u, v, w)
            b = loc.loc_belief(h)
            close(b, ref.B)
            assert (b[:, occ != 0] == 0.0).all()
    finally:
        loc.loc_destroy(h)


def test_tiled_restart_after_all_mass_removed():
    occ = np.ones((40, 64), np.uint8)
    occ[18:22, 30:34] = 0
    h = make(occ, 8, 1.0)
    try:
        loc.loc_step(h, 12.0, 0.0, 0.0)                # everything walks into walls
        st = loc.loc_stats(h)
        b = loc.loc_belief(h)
        assert st["n_reinit"] == 1 and st["last_Z"] == 0.0
        M = (occ == 0).astype(np.float64)
        assert np.abs(b - F.uniform_belief(M, 8)).max() <= 1e-9
        loc.loc_step(h, 0.0, 0.0, 0.0)                 # the next step starts from uniform
        ref = F.Filter(occ, 8, 1.0)
        ref.step(0.0, 0.0, 0.0)
        close(loc.loc_belief(h), ref.B)
    finally:
        loc.loc_destroy(h)


def test_tiled_is_refused_where_it_does_not_apply():
    occ = np.zeros((32, 30), np.uint8)                 # W * 4 bytes not a multiple of 16
    with pytest.raises(loc.LocError):
        make(occ, 16, 0.1)
    with pytest.raises(loc.LocError):
        make(np.zeros((32, 32), np.uint8), 6, 0.1)    # K below the tiled minimum
    with pytest.raises(loc.LocError):
        make(np.zeros((32, 32), np.uint8), 16, 0.1, sigma_xy_cells=1.0)
    with pytest.raises(loc.LocError):
        make(np.zeros((32, 32), np.uint8), 16, 0.1, tile=19)   # beyond LOC_TILE_CONFIGS


@pytest.mark.parametrize("storage", ["bf16", "f16"])
def test_reduced_precision_trajectory_l1_and_argmax(storage):
    """Reduced-precision storage (FP32 arithmetic; BF16 rounded by error diffusion along theta, FP16 scaled by
    2^14): L1 <= 1e-2 against the FP64 oracle over the whole 200-step trajectory, and the same
    argmax bin wherever the oracle's maximum is unambiguous."""
    wl = workloads.get("rooms64")
    occ = workloads.make_map(wl)
    walk = workloads.make_walk(wl, occ)
    h = make(occ, wl["K"], wl["cell"], storage=storage)
    ref = F.Filter(occ, wl["K"], wl["cell"])
    worst = 0.0
    try:
        for t, (u, v, w) in enumerate(walk.odom, start=1):
            loc.loc_step(h, u, v, w)
            ref.step(u, v, w)
            if t % 25 == 0:
                b = loc.loc_belief(h).astype(np.float64)
                l1 = np.abs(b - ref.B).sum()
                worst = max(worst, l1)
                assert l1 <= 1e-2, (t, l1)
                k, j, i, p = R.argmax_pose(ref.B)
                top2 = np.sort(ref.B.reshape(-1))[-2:]
                if top2[1] - top2[0] > 2 * 1e-2 * top2[1]:
                    assert loc.loc_argmax(h)[:3] == (k, j, i), t
    finally:
        loc.loc_destroy(h)
    print(f"{storage}: worst L1 over the trajectory {worst:.3e}")


@pytest.mark.parametrize("storage", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("packed,scalar", [(14, 6), (15, 13)])
def test_split_producers_are_bit_identical(packed, scalar, storage):
    """Split producers (S warps beside X warps) run the same passes on the same cells as the
    configuration with the same tile rows and consumer layout: bit-identical tensors and
    normalisers, step after step, including the BF16 rounding residuals carried along theta."""
    H, W, K = 75, 200, 20
    rng = np.random.default_rng(packed)
    occ = (rng.random((H, W)) < 0.15).astype(np.uint8)
    b = fields.belief_like(occ, K, seed=packed, dtype=np.float32)
    hp = make(occ, K, 0.05, tile=packed, storage=storage)
    hs = make(occ, K, 0.05, tile=scalar, storage=storage)
    try:
        loc.loc_set_belief(hp, b)
        loc.loc_set_belief(hs, b)
        for (u, v, w) in [(0.013, -0.041, 0.05), (0.07, 0.02, -0.1), (-0.11, 0.09, 0.0)]:
            loc.loc_step(hp, u, v, w)
            loc.loc_step(hs, u, v, w)
            assert np.array_equal(loc.loc_belief(hp), loc.loc_belief(hs))
            assert loc.loc_stats(hp)["last_Z"] == loc.loc_stats(hs)["last_Z"]
    finally:
        loc.loc_destroy(hp)
        loc.loc_destroy(hs)


@pytest.mark.parametrize("storage", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("piped,plain", [(17, 3), (18, 2)])
def test_pipelined_tiles_are_bit_identical(piped, plain, storage):
    """The software-pipelined configurations (the S-pass of plane p, the X-pass of p - 1 and the
    P-pass of p - 2 between one barrier) run the same passes on the same cells as the synchronous
    configuration with the same tile: bit-identical tensors and normalisers, step after step,
    including a restart read from the map."""
    H, W, K = 75, 200, 20
    rng = np.random.default_rng(piped)
    occ = (rng.random((H, W)) < 0.15).astype(np.uint8)
    b = fields.belief_like(occ, K, seed=piped, dtype=np.float32)
    hp = make(occ, K, 0.05, tile=piped, storage=storage)
    hs = make(occ, K, 0.05, tile=plain, storage=storage)
    try:
        for (u, v, w) in [(0.02, 0.01, 0.0)]:          # the first step reads the uniform start
            loc.loc_step(hp, u, v, w)
            loc.loc_step(hs, u, v, w)
            assert np.array_equal(loc.loc_belief(hp), loc.loc_belief(hs))
        loc.loc_set_belief(hp, b)
        loc.loc_set_belief(hs, b)
        for (u, v, w) in [(0.013, -0.041, 0.05), (0.07, 0.02, -0.1), (-0.11, 0.09, 0.0)]:
            loc.loc_step(hp, u, v, w)
            loc.loc_step(hs, u, v, w)
            assert np.array_equal(loc.loc_belief(hp), loc.loc_belief(hs))
            assert loc.loc_stats(hp)["last_Z"] == loc.loc_stats(hs)["last_Z"]
    finally:
        loc.loc_destroy(hp)
        loc.loc_destroy(hs)


FUSED = [6, 7, 13, 14, 15, 16]                  # the warp-specialised configurations
UNFUSED = [1, 3, 8]                             # synchronous and paired: the pass after the step


def full_pass_argmax(h):
    """The argmax pass over the stored tensor (loc_estimate runs it before its own pass)."""
    e = loc.loc_estimate(h, 0.0, 0)
    return (e["k"], e["j"], e["i"]), e["p"]


@pytest.mark.parametrize("storage", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("tile", FUSED + UNFUSED)
def test_fused_argmax_equals_the_argmax_pass(tile, storage):
    """After a warp-specialised propagation loc_argmax reads the argmax the step kernel itself
    combined (per-thread running maxima of the stored values, lowest index on ties): the same
    state and value as the separate pass over the stored tensor, step after step.  The other
    configurations take the pass, with the same results."""
    H, W, K = 75, 200, 20
    rng = np.random.default_rng(100 + tile)
    occ = (rng.random((H, W)) < 0.15).astype(np.uint8)
    b = fields.belief_like(occ, K, seed=tile, dtype=np.float32)
    h = make(occ, K, 0.05, tile=tile, storage=storage)
    try:
        loc.loc_set_belief(h, b)
        for (u, v, w) in [(0.013, -0.041, 0.05), (0.07, 0.02, -0.1), (-0.11, 0.09, 0.0), (0.0, 0.0, 0.0)]:
            loc.loc_step(h, u, v, w)
            got = loc.loc_argmax(h)
            want, p = full_pass_argmax(h)
            assert got[:3] == want
            assert abs(got[3] - p) <= 1e-6 * p
            assert loc.loc_argmax(h) == got            # a second read: the same result
    finally:
        loc.loc_destroy(h)


@pytest.mark.parametrize("storage", ["f32", "bf16"])
@pytest.mark.parametrize("tile", [3, 6, 14, 15, 16])
def test_fused_argmax_ties_and_restart(tile, storage):
    """Exact ties: a uniform belief on a free map stepped without motion leaves every interior
    cell with the bit-identical value, so the lowest [K][H][W] index among the maxima must win.
    A step that removes all mass restarts the session; loc_argmax then falls back to the pass
    over the uniform restart state (the first free cell of bin 0)."""
    H, W, K = 60, 128, 12
    occ = np.zeros((H, W), np.uint8)
    h = make(occ, K, 0.1, tile=tile, storage=storage)
    try:
        loc.loc_set_belief(h, np.ones((K, H, W), np.float32))
        loc.loc_step(h, 0.0, 0.0, 0.0)
        got = loc.loc_argmax(h)
        want, p = full_pass_argmax(h)
        assert got[:3] == want and abs(got[3] - p) <= 1e-6 * p
        flat = loc.loc_belief(h).reshape(-1)
        assert (flat == flat.max()).sum() > 1               # ties exist
    finally:
        loc.loc_destroy(h)
    occ = np.ones((40, 64), np.uint8)
    occ[18:22, 30:34] = 0
    h = make(occ, 8, 1.0, tile=tile, storage=storage)
    try:
        loc.loc_step(h, 12.0, 0.0, 0.0)                 # everything walks into walls
        assert loc.loc_stats(h)["n_reinit"] == 1
        k, j, i, p = loc.loc_argmax(h)
        assert (k, j, i) == (0, 18, 30)
        assert abs(p - 1.0 / (8 * 16)) <= 1e-6 / (8 * 16)
    finally:
        loc.loc_destroy(h)
