"""GPU parity of loc_estimate (the pose estimate, the belief near it and the second hypothesis)
against ``oracle.readout.estimate``.

Both passes are covered: one thread per cell (a grid whose H W is not a multiple of the 16-byte
group) and the flat 16-byte pass.  The argmax state and the second hypothesis's cell are exact
(the belief values are distinct);
the near mass agrees to 1e-6 relative; the second value to FP32 rounding of the stored belief.
"""
import math

import numpy as np
import pytest

import paper_1910_00572_gb300 as loc
from oracle import readout as R
from synth import fields, floorplan, trajectory

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1910_00572_gb300 import build
    build.build()
    loc.lib()


def compare(got, want):
    assert (got["k"], got["j"], got["i"]) == (want["k"], want["j"], want["i"])
    assert (got["second_j"], got["second_i"]) == (want["second_j"], want["second_i"])
    assert abs(got["mass_near"] - want["mass_near"]) <= 1e-6 * max(want["mass_near"], 1e-30) + 1e-12
    assert abs(got["p"] - want["p"]) <= 1e-6 * want["p"]
    assert abs(got["second_p"] - want["second_p"]) <= 1e-6 * want["second_p"] + 1e-15
    for key in ("x", "y", "theta"):
        assert abs(got[key] - want[key]) <= 1e-9, key


@pytest.mark.parametrize("H,W", [(50, 61), (48, 64)], ids=["per-cell pass", "16-byte pass"])
@pytest.mark.parametrize("storage", ["f32", "bf16"])
@pytest.mark.parametrize("radius,dk", [(0.0, 0), (0.3, 1), (1.0, 3), (50.0, 64)])
def test_estimate_matches_oracle(H, W, storage, radius, dk):
    occ = floorplan.rooms_map(3, size=64)[:H, :W].copy()
    K, cell = 16, 0.1
    b = fields.belief_like(occ, K, seed=7, dtype=np.float32)
    p = loc.loc_params_default(H=H, W=W, K=K, cell_m=cell, storage=storage)
    h = loc.loc_create(occ, p)
    try:
        loc.loc_set_belief(h, b)
        ref = loc.loc_belief(h).astype(np.float64)     # the stored belief, as the oracle's input
        got = loc.loc_estimate(h, radius, dk)
        st = loc.loc_stats(h)
    finally:
        loc.loc_destroy(h)
    compare(got, R.estimate(ref, cell, st["theta"], radius, dk))


def test_estimate_after_steps_and_the_restart_state():
    occ = floorplan.rooms_map(4, size=48)
    K, cell = 8, 0.1
    walk = trajectory.random_walk(occ, cell, 5, 0.1, 3)
    h = loc.loc_create(occ, loc.loc_params_default(H=48, W=48, K=K, cell_m=cell))
    try:
        e0 = loc.loc_estimate(h, 0.5, 2)                # uniform: ties go to the lowest index
        ref0 = R.estimate(loc.loc_belief(h).astype(np.float64), cell, 0.0, 0.5, 2)
        assert (e0["k"], e0["j"], e0["i"]) == (ref0["k"], ref0["j"], ref0["i"])
        assert (e0["second_j"], e0["second_i"]) == (ref0["second_j"], ref0["second_i"])
        for u, v, w in walk.odom:
            loc.loc_step(h, u, v, w)
        b = loc.loc_belief(h).astype(np.float64)
        compare(loc.loc_estimate(h, 0.5, 2), R.estimate(b, cell, loc.loc_stats(h)["theta"], 0.5, 2))
        with pytest.raises(loc.LocError):
            loc.loc_estimate(h, -1.0, 0)
        with pytest.raises(loc.LocError):
            loc.loc_estimate(h, math.nan, 0)
        with pytest.raises(loc.LocError):
            loc.loc_estimate(h, 1.0, -1)
    finally:
        loc.loc_destroy(h)
