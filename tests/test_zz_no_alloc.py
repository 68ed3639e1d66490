"""The allocation-free propagation entry point, for callers that cannot allocate device
memory while they run (real-time loops, stacks with memory fixed at start-up, hosts whose
allocator belongs to another runtime).  Through the C-ABI, two calls in a row must match
the session API's propagation (the existing entry point) within the parity tolerance used by
the other GPU tests.  This file is collected last on purpose."""
import numpy as np
import pytest

import paper_1910_00572_gb300 as loc
from synth import fields, floorplan

pytestmark = pytest.mark.gpu

ABS_TOL = 1e-6
REL_TOL = 2e-5


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1910_00572_gb300 import build
    build.build()
    loc.lib()


def _occ(H, W, seed):
    """An office-plan crop of H x W cells (a larger plan when the crop needs it)."""
    side = max(256, 1 << (max(H, W) - 1).bit_length())
    big = floorplan.office_map(seed, size=side)
    return floorplan.crop(big, (side - H) // 2, (side - W) // 2, H, W)


# (H, W, K, sigma_xy_cells, sigma_theta_bins): the office crop of the first version; ragged H
# and W (multiples of neither the 16-row nor the 32-column tile); no x/y blur (radius 0);
# K = 4 with a theta radius of 4 (the ring of 9 planes wraps the 4 bins more than once); and
# 2048 x 2048 cells, exactly the 8192 tiles the scratch array holds.
CASES = [
    (96, 112, 12, 0.5, 1.0),
    (101, 75, 12, 0.5, 1.0),
    (96, 112, 12, 0.0, 1.0),
    (80, 72, 4, 0.5, 1.2),
    (2048, 2048, 2, 0.5, 1.0),
]


@pytest.mark.parametrize("H,W,K,sxy,sth", CASES, ids=[f"{c[0]}x{c[1]}x{c[2]}_s{c[3]}_{c[4]}" for c in CASES])
def test_noalloc_matches_session_step_twice(H, W, K, sxy, sth):
    import torch
    occ = _occ(H, W, 7)
    cell = 0.05
    b = fields.belief_like(occ, K, seed=3, dtype=np.float32)
    dev = torch.device("cuda", 0)
    p = loc.loc_params_default(H=H, W=W, K=K, cell_m=cell, sigma_xy_cells=sxy, sigma_theta_bins=sth,
                               stream=loc.torch_stream())
    occ_d = torch.from_numpy(occ).to(dev)
    cur = torch.from_numpy(b).to(dev)
    out = torch.empty_like(cur)
    z = torch.zeros(1, dtype=torch.float64, device=dev)
    h = loc.loc_create(occ, p)
    try:
        loc.loc_set_belief(h, b)
        for (dx, dy) in [(0.031, -0.017), (-0.02, 0.045)]:
            loc.loc_propagate_noalloc(p, occ_d.data_ptr(), cur.data_ptr(), out.data_ptr(),
                                      z.data_ptr(), dx, dy)
            torch.cuda.synchronize()
            in_sum = float(cur.double().sum())
            loc.loc_step(h, dx, dy, 0.0)              # heading offset stays 0: same frame
            want = loc.loc_belief(h).astype(np.float64)
            zz = float(z.item())
            got = out.cpu().numpy().astype(np.float64) / zz
            err = np.abs(got - want).max()
            assert err <= ABS_TOL and err <= REL_TOL * want.max(), err
            assert abs(zz / in_sum - loc.loc_stats(h)["last_Z"]) <= 1e-6
            assert abs(zz - float(out.double().sum())) <= 1e-6 * zz
            cur, out = out, cur
    finally:
        loc.loc_destroy(h)


def test_noalloc_rejects_grids_beyond_the_scratch():
    import torch
    dev = torch.device("cuda", 0)
    small = torch.zeros(16, dtype=torch.float32, device=dev)
    z = torch.zeros(1, dtype=torch.float64, device=dev)
    p = loc.loc_params_default(H=4096, W=4096, K=8, cell_m=0.05)
    with pytest.raises(loc.LocError) as e:
        loc.loc_propagate_noalloc(p, small.data_ptr(), small.data_ptr(), small.data_ptr(),
                                  z.data_ptr(), 0.01, 0.0)
    assert e.value.status == loc.LOC_ERR_INVALID_ARG
    assert "8192" in loc.loc_last_error()
