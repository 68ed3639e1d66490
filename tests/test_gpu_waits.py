"""Failure detection of the bounded device waits, without a GPU fault.

The Floyd-Steinberg block hand-offs of the scan update poll a progress flag in global memory
with a bounded wait.  The test hook loc_debug_fs_stall makes every hand-off wait on a flag
that nothing sets, with a 10 ms limit: the kernel must give up, record the timeout in the
session's status and return.  The host then reports LOC_ERR_TIMEOUT, the handle stays failed
(LOC_ERR_STATE on every later call), and the CUDA context stays usable: a fresh session on
the same device still matches the oracle.  Nothing faults, traps or hangs."""
import math

import numpy as np
import pytest

import paper_1910_00572_gb300 as loc
from oracle import filter as F
from synth import floorplan, scan

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1910_00572_gb300 import build
    build.build()
    loc.lib()


def test_dithering_wait_runs_out_and_fails_the_handle_only():
    occ = floorplan.office_map(5, size=256)[:160, :192].copy()
    occ[0, :] = occ[-1, :] = 1
    occ[:, 0] = occ[:, -1] = 1
    H, W, K, cell = occ.shape[0], occ.shape[1], 8, 0.05
    free = np.argwhere(occ == 0)[len(np.argwhere(occ == 0)) // 2]
    pose = ((free[1] + 0.5) * cell, (free[0] + 0.5) * cell, 0.3)
    z = scan.simulate_scan(occ, cell, pose, seed=1, n_beams=360, r_max=10.0, noise_sigma=0.05, dropout=0.05)
    p = loc.loc_params_default(H=H, W=W, K=K, cell_m=cell, n_samples=512)
    h = loc.loc_create(occ, p)
    try:
        loc.loc_step(h, 0.02, 0.01, 0.0)
        loc.loc_lidar_update(h, z, 0.0, math.pi / 180, 10.0, 4, 0.1)     # a normal scan first
        loc.loc_sync(h)
        loc.loc_debug_fs_stall(True, 0.01)
        try:
            loc.loc_lidar_update(h, z, 0.0, math.pi / 180, 10.0, 4, 0.1)   # launches; the waits give up
            with pytest.raises(loc.LocError) as e:
                loc.loc_sync(h)
            assert e.value.status == loc.LOC_ERR_TIMEOUT
        finally:
            loc.loc_debug_fs_stall(False, 0.2)
        for call in (lambda: loc.loc_step(h, 0.01, 0.0, 0.0), lambda: loc.loc_belief(h), lambda: loc.loc_sync(h)):
            with pytest.raises(loc.LocError) as e:
                call()
            assert e.value.status == loc.LOC_ERR_STATE             # sticky until destroy
    finally:
        loc.loc_destroy(h)
    # the context is intact: a new session on the same device propagates and matches the oracle
    h2 = loc.loc_create(occ, p)
    ref = F.Filter(occ, K, cell)
    try:
        for (u, v, w) in [(0.03, -0.01, 0.02), (0.0, 0.04, -0.01)]:
            loc.loc_step(h2, u, v, w)
            ref.step(u, v, w)
        assert np.abs(loc.loc_belief(h2).astype(np.float64) - ref.B).max() <= 1e-6
        loc.loc_lidar_update(h2, z, 0.0, math.pi / 180, 10.0, 4, 0.1)   # dithering works again
        loc.loc_sync(h2)
        assert loc.loc_samples(h2).size > 0
    finally:
        loc.loc_destroy(h2)


def test_debug_hook_arguments():
    with pytest.raises(loc.LocError) as e:
        loc.loc_debug_fs_stall(True, 0.0)
    assert e.value.status == loc.LOC_ERR_INVALID_ARG
    with pytest.raises(loc.LocError):
        loc.loc_debug_fs_stall(False, 11.0)
