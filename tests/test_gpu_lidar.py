"""GPU parity of the LIDAR sample update (Section III-B) through the C-ABI.

* Floyd-Steinberg selection and the ray-cast expected ranges decide integers, so both are
  compared bit for bit with the oracle's FP32 implementations on the same inputs.
* The likelihood and the Eq. 9 reweighting of a given sample set are compared with the FP64
  oracle within 1e-6 absolute and 2e-5 of the largest value (FP32 log-likelihoods: the
  states that keep weight have |log L| of order 10, where FP32 is good to ~1e-6).
* loc_lidar_update with the GPU's own dithering is checked by properties that hold for any
  valid selection: the belief still sums to 1, unsampled states are untouched, the number of
  samples follows the Floyd-Steinberg count bound, and the true pose gains weight.
"""
import math

import numpy as np
import pytest

import paper_1910_00572_gb300 as loc
from oracle import cprop
from oracle import filter as F
from oracle import lidar as OL
from oracle import readout as R
from synth import fields, floorplan, scan, workloads

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


# ------------------------------------------------------------------ Floyd-Steinberg

@pytest.mark.parametrize("H,W,n_s", [(5, 7, 6), (64, 64, 300), (100, 37, 500), (300, 257, 4096),
                                     (97, 1100, 2000), (2048, 2048, 4096), (4200, 96, 3000)])
def test_dithering_is_bit_exact(H, W, n_s):
    """Bit-exact against the oracle's FP32 C code, from a handful of cells to 2048 x 2048 and
    4200 rows (132 row blocks, so each of the 16 warps takes eight or nine blocks)."""
    m = fields.map_like(H, W, seed=H + W)
    fs = float(OL.fs_factor(m, n_s))
    h = make(np.zeros((H, W), np.uint8), 8, 0.05)
    try:
        sel, count = loc.loc_dither(h, m, fs)
    finally:
        loc.loc_destroy(h)
    want = OL.fs_select(m, fs)
    assert count == int(want.sum())
    assert np.array_equal(sel, want)


def test_dithering_half_grey_checkerboard():
    h = make(np.zeros((40, 72), np.uint8), 8, 0.05)
    try:
        sel, _ = loc.loc_dither(h, np.full((40, 72), 0.5, np.float32), 1.0)
    finally:
        loc.loc_destroy(h)
    J, I = np.mgrid[0:40, 0:72]
    assert (sel == ((I + J) % 2 == 0)).all()


# ------------------------------------------------------------------ ray casting

def test_ray_ranges_are_bit_exact():
    occ = floorplan.crop(floorplan.office_map(3, size=512), 100, 60, 256, 256)
    rng = np.random.default_rng(0)
    free = np.flatnonzero(occ.reshape(-1) == 0)
    cells = rng.choice(free, 300, replace=False).astype(np.int32)
    cells = np.append(cells, np.flatnonzero(occ.reshape(-1) != 0)[:5]).astype(np.int32)  # occupied: 0
    ang = np.concatenate([rng.uniform(-math.pi, math.pi, 200), np.arange(8) * math.pi / 4])
    dirs = OL.beam_dirs32(ang)
    h = make(occ, 8, 0.05)
    try:
        got = loc.loc_ray_ranges(h, cells, dirs, 10.0)
    finally:
        loc.loc_destroy(h)
    want = OL.expected_ranges(occ, cells, dirs, 10.0, 0.05)
    assert np.array_equal(got, want)


# ------------------------------------------------------------------ Eq. 9 on a given set

def lidar_case(seed, storage="f32", K=16, size=96, n_samples=400):
    occ = floorplan.crop(floorplan.office_map(seed, size=256), 30, 40, size, size)
    cell = 0.05
    rng = np.random.default_rng(seed)
    free = np.argwhere(occ == 0)
    j, i = free[rng.integers(len(free))]
    theta = 0.37
    k_true = 5
    pose = ((i + 0.5) * cell, (j + 0.5) * cell, 2 * math.pi * k_true / K + theta)
    z = scan.simulate_scan(occ, cell, pose, seed=seed, n_beams=360, r_max=4.0, noise_sigma=0.02)
    b = fields.belief_like(occ, K, seed=seed, dtype=np.float32)
    return occ, cell, theta, z, b, (k_true, j, i)


@pytest.mark.parametrize("seed", [1, 2])
def test_reweight_with_given_cells_matches_oracle(seed):
    occ, cell, theta, z, b, _ = lidar_case(seed)
    K = b.shape[0]
    b64 = b.astype(np.float64) / b.astype(np.float64).sum()
    m32 = b64.max(axis=0).astype(np.float32)
    cells = OL.samples_from_mask(OL.fs_select(m32, OL.fs_factor(m32, 400)))
    assert cells.size > 50
    h = make(occ, K, cell)
    try:
        loc.loc_set_belief(h, b)
        loc.loc_step(h, 0.0, 0.0, theta)              # heading offset theta_t = theta (no motion:
        ref = F.Filter(occ, K, cell)                 # the propagation is the blur only)
        ref.B = b64.copy()
        ref.step(0.0, 0.0, theta)
        before = loc.loc_belief(h)
        loc.loc_lidar_update_cells(h, cells, z, 0.0, math.pi / 180, 4.0, 4, 0.1)
        got = loc.loc_belief(h)
        st = loc.loc_stats(h)
    finally:
        loc.loc_destroy(h)
    want, _ = OL.lidar_update(ref.B, occ, theta, z, cell, 0.0, math.pi / 180, 4.0, 4, 0.1, 400, cells=cells)
    err = np.abs(got.astype(np.float64) - want).max()
    assert err <= ABS_TOL and err <= REL_TOL * want.max(), err
    flat_b, flat_g = before.reshape(K, -1), got.reshape(K, -1)
    others = np.setdiff1d(np.arange(flat_b.shape[1]), cells)
    assert np.array_equal(flat_b[:, others] * 1.0, flat_g[:, others] * 1.0) or \
        np.abs(flat_b[:, others] - flat_g[:, others]).max() <= 1e-7 * flat_b.max()
    assert abs(got.astype(np.float64).sum() - 1.0) < 1e-5


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_reweight_when_the_scan_disagrees_with_the_belief(storage):
    """A scan taken far from where the belief lies: the sampled set holds cells of the scan's
    pose (zero belief, where the likelihood peaks) and cells of the belief (log-likelihoods
    about 9500 below the maximum).  Eq. 9 still moves the set's mass onto its best states with
    belief, finite, as the oracle does; before the weights were normalised in the log domain
    their sum underflowed (a served session's normaliser became non-finite).  The device sums
    each log-likelihood in FP32, good to about 1e-3 absolute at these magnitudes, so the
    result is checked by L1 and the argmax state rather than element by element."""
    occ = floorplan.office_map(6, size=256)[40:200, 30:210].copy()
    occ[0, :] = occ[-1, :] = 1
    occ[:, 0] = occ[:, -1] = 1
    H, W = occ.shape
    K, cell, theta = 16, 0.05, 0.0
    free = np.argwhere(occ == 0)
    rng = np.random.default_rng(4)
    a = free[np.argmin(np.abs(free[:, 0] - 20) + np.abs(free[:, 1] - 20))]     # belief here
    c = free[np.argmin(np.abs(free[:, 0] - 140) + np.abs(free[:, 1] - 160))]   # scan from here
    b = np.zeros((K, H, W), np.float32)
    b[:, max(0, a[0] - 3):a[0] + 4, max(0, a[1] - 3):a[1] + 4] = rng.random((K, 7, 7)).astype(np.float32)
    b[:, occ != 0] = 0.0
    b /= b.sum()
    z = scan.simulate_scan(occ, cell, ((c[1] + 0.5) * cell, (c[0] + 0.5) * cell, 0.0), seed=3, n_beams=360,
                           r_max=10.0, noise_sigma=0.02)
    near_a = [(j, i) for j in range(a[0] - 3, a[0] + 4) for i in range(a[1] - 3, a[1] + 4)
              if 0 <= j < H and 0 <= i < W and occ[j, i] == 0]
    near_c = [(j, i) for j in range(c[0] - 2, c[0] + 3) for i in range(c[1] - 2, c[1] + 3)
              if 0 <= j < H and 0 <= i < W and occ[j, i] == 0]
    cells = np.array(sorted(j * W + i for j, i in near_a + near_c), np.int32)
    h = make(occ, K, cell, storage=storage, sigma_xy_cells=0.0, sigma_theta_bins=0.0)
    try:
        loc.loc_set_belief(h, b)
        before = loc.loc_belief(h).astype(np.float64)
        loc.loc_lidar_update_cells(h, cells, z, 0.0, math.pi / 180, 10.0, 4, 0.1)
        loc.loc_sync(h)
        got = loc.loc_belief(h).astype(np.float64)
    finally:
        loc.loc_destroy(h)
    assert np.all(np.isfinite(got))
    want, _ = OL.lidar_update(before, occ, theta, z, cell, 0.0, math.pi / 180, 10.0, 4, 0.1, 0, cells=cells)
    assert abs(got.sum() - 1.0) < 1e-4
    # the set's mass left the scan's pose for the belief's states, as the oracle's does
    assert np.abs(got - want).sum() <= 1e-2
    assert np.unravel_index(np.argmax(got), got.shape) == np.unravel_index(np.argmax(want), want.shape)


def test_lidar_update_properties_with_device_dithering():
    occ, cell, theta, z, b, (k_true, j_true, i_true) = lidar_case(4, n_samples=600)
    K = b.shape[0]
    p = loc.loc_params_default(H=occ.shape[0], W=occ.shape[1], K=K, cell_m=cell, n_samples=600)
    h = loc.loc_create(occ, p)
    try:
        loc.loc_set_belief(h, b)
        loc.loc_step(h, 0.0, 0.0, theta)
        before = loc.loc_belief(h)
        m_before = loc.loc_marginal(h, loc.LOC_MAP_MAX)
        loc.loc_lidar_update(h, z, 0.0, math.pi / 180, 4.0, 4, 0.1)
        got = loc.loc_belief(h)
        cells = loc.loc_samples(h)
    finally:
        loc.loc_destroy(h)
    H, W = occ.shape
    v = np.minimum(1.0, 600 * m_before.astype(np.float64) / m_before.astype(np.float64).sum())
    assert abs(cells.size - v.sum()) <= H + W
    assert np.all(np.diff(cells) > 0)                                  # raster order, unique
    flat_b, flat_g = before.reshape(K, -1), got.reshape(K, -1)
    others = np.setdiff1d(np.arange(H * W), cells)
    assert np.abs(flat_b[:, others] - flat_g[:, others]).max() <= 1e-7 * flat_b.max()
    assert abs(flat_g[:, cells].sum() - flat_b[:, cells].sum()) <= 1e-5
    assert abs(got.astype(np.float64).sum() - 1.0) < 1e-5


# ------------------------------------------------------------------ trajectories with scans

def run_lidar_trajectory(storage, size, K, steps, scan_every, seed, check):
    """A walk on a size x size office crop with a scan every scan_every-th step, on the GPU and
    on the oracle in lockstep; the scan's sample set is the oracle's Floyd-Steinberg selection
    (replayed on the GPU through loc_lidar_update_cells).  check(t, got, want) runs after every
    scan with the normalised GPU and oracle tensors.  The oracle propagates through its C
    restatement (bit-identical to the numpy definition) on all host cores."""
    wl = workloads.get("office2048")
    occ = floorplan.crop(floorplan.office_map(seed, size=1024), 300, 280, size, size)
    cell = 0.05
    walk = workloads.make_walk(dict(wl, seed=seed), occ, steps=steps)
    p = loc.loc_params_default(H=size, W=size, K=K, cell_m=cell, storage=storage)
    h = loc.loc_create(occ, p)
    ref = cprop.Filter(occ, K, cell, threads=cprop.host_cores())
    try:
        for t, (u, v, w) in enumerate(walk.odom, start=1):
            loc.loc_step(h, u, v, w)
            ref.step(u, v, w)
            if t % scan_every == 0:
                z = scan.simulate_scan(occ, cell, walk.poses[t], seed=seed * 7919 + t, n_beams=360,
                                       r_max=10.0, noise_sigma=0.05, dropout=0.05)
                m32 = ref.B.max(axis=0).astype(np.float32)
                cells = OL.samples_from_mask(OL.fs_select(m32, OL.fs_factor(m32, 1024)))
                loc.loc_lidar_update_cells(h, cells, z, 0.0, math.pi / 180, 10.0, 4, 0.1)
                ref.B, _ = OL.lidar_update(ref.B, occ, ref.odo.theta, z, cell, 0.0, math.pi / 180,
                                           10.0, 4, 0.1, 1024, cells=cells)
                check(t, loc.loc_belief(h).astype(np.float64), ref.B)
    finally:
        loc.loc_destroy(h)
    return walk


def test_fp32_trajectory_with_scans_matches_oracle():
    """FP32 storage, 60 steps with 6 scans: 1e-6 absolute and 2e-5 of the tensor's maximum, the
    bars of the plain propagation (the sampled states' FP32 log-likelihoods differ from the
    FP64 ones by about 1e-6 relative of |log L|, and the states that keep weight have |log L -
    max log L| of order 10)."""
    def check(t, got, want):
        err = np.abs(got - want).max()
        assert err <= ABS_TOL and err <= REL_TOL * want.max(), (t, err, err / want.max())
    run_lidar_trajectory("f32", 96, 16, 60, 10, seed=11, check=check)


def crop_trajectory_l1(storage):
    """Config 2's parity run as specified: the 256 x 256 crop, 72 bins, 1000 steps with a scan
    every 10th step (100 scans).  Returns the L1 distance to the FP64 oracle after every scan
    and checks the argmax state there whenever the oracle's top two states differ by more than
    2 % (else the argmax is ambiguous at reduced precision)."""
    curve = []

    def check(t, got, want):
        curve.append((t, float(np.abs(got - want).sum())))
        top2 = np.partition(want.reshape(-1), -2)[-2:]
        if top2[1] - top2[0] > 2e-2 * top2[1]:
            assert np.unravel_index(np.argmax(got), got.shape) == np.unravel_index(np.argmax(want), want.shape), t
    run_lidar_trajectory(storage, 256, 72, 1000, 10, seed=2, check=check)
    assert len(curve) == 100
    print(f"{storage} crop L1 curve (step:L1):", " ".join(f"{t}:{l1:.2e}" for t, l1 in curve))
    return np.array([l1 for _, l1 in curve])


@pytest.mark.slow
def test_f16_crop_trajectory_with_scans_meets_the_l1_bar():
    """FP16 storage (11 significant bits, the 2^14 multiplier): L1 <= 1e-2 at every one of the
    100 checkpoints (measured: below 1e-3)."""
    l1 = crop_trajectory_l1("f16")
    assert l1.max() <= 1e-2, l1.max()


@pytest.mark.slow
def test_bf16_crop_trajectory_with_scans_l1_and_argmax():
    """BF16 storage on the same trajectory: L1 <= 1e-2 at every one of the 100 checkpoints,
    besides the argmax.  The stored values keep 8 significant bits.  Rounded independently
    (stochastic rounding, unbiased per value), a hypothesis whose mass sits in a few states
    random-walks that mass by about 2^-8 sqrt(t / (6 n_eff)) relative after t steps, and a scan
    that weighs two such hypotheses turns the difference into L1: on this run it passed 1e-2 at
    15 checkpoints.  The kernels round by error diffusion along theta instead (each cell's
    residual carried from bin to bin), which keeps every cell's mass over its bins to within
    half a unit in the last place, step after step, so the mass no longer random-walks."""
    l1 = crop_trajectory_l1("bf16")
    assert l1.max() <= 1e-2, (l1.max(), int(np.argmax(l1)))
