"""The C-ABI library loads on a machine without a GPU and exports every function that the
headers in include/ declare (no compute calls here)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(loc_\w+)\s*\(", src, flags=re.M):
            if "typedef" not in m.group(0) and "(*" not in m.group(0):
                names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def libloc():
    from paper_1910_00572_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_headers_declare_the_session_api():
    names = declared_functions()
    for n in ("loc_create", "loc_step", "loc_belief", "loc_marginal", "loc_destroy"):
        assert n in names


def test_library_exports_every_declared_function(libloc):
    missing = [n for n in declared_functions() if not hasattr(libloc, n)]
    assert not missing, missing


def test_invalid_arguments_fail_without_gpu_work(libloc):
    import paper_1910_00572_gb300 as loc
    import numpy as np
    p = loc.loc_params_default(H=0, W=4, K=4, cell_m=0.1)
    with pytest.raises(loc.LocError) as e:
        loc.loc_create(np.zeros((0, 4), np.uint8), p)
    assert e.value.status == loc.LOC_ERR_INVALID_ARG
    p = loc.loc_params_default(H=4, W=4, K=4, cell_m=0.1)
    with pytest.raises(loc.LocError) as e:
        loc.loc_create(np.ones((4, 4), np.uint8), p)          # no free cell
    assert e.value.status == loc.LOC_ERR_INVALID_ARG
    assert "free" in loc.loc_last_error()
    p = loc.loc_params_default(H=4, W=4, K=4, cell_m=0.1, sigma_xy_cells=5.0)
    with pytest.raises(loc.LocError):
        loc.loc_create(np.zeros((4, 4), np.uint8), p)          # radius 15 > LOC_MAX_R_XY


def test_batch_arguments_fail_without_gpu_work(libloc):
    import paper_1910_00572_gb300 as loc
    with pytest.raises(loc.LocError) as e:
        loc.loc_batch_create([])
    assert e.value.status == loc.LOC_ERR_INVALID_ARG
    assert "no sessions" in loc.loc_last_error()
    with pytest.raises(loc.LocError) as e:
        loc.loc_batch_step(loc.Batch(0, []), [], [], [])
    assert e.value.status == loc.LOC_ERR_INVALID_ARG
    assert loc.loc_batch_destroy(None) is None


def test_server_and_admission_arguments_fail_without_gpu_work(libloc):
    import paper_1910_00572_gb300 as loc
    for kw in (dict(hbm_budget_bytes=0.0), dict(storage=7), dict(tile=9), dict(n_streams=0)):
        with pytest.raises(loc.LocError) as e:
            loc.loc_server_create(loc.loc_server_params_default(**kw))
        assert e.value.status == loc.LOC_ERR_INVALID_ARG
    p = loc.loc_params_default(H=100, W=60, K=8, cell_m=0.05, storage="bf16", n_samples=0)
    b = loc.loc_session_bytes(p)
    # two 16-bit belief tensors, the map, the correction and the sampling scratch
    assert b >= 2 * 2 * 100 * 60 * 8 + 100 * 60 * (1 + 4 + 4 + 1)
    p.K = 0
    with pytest.raises(loc.LocError):
        loc.loc_session_bytes(p)


def test_anisotropic_arguments_fail_without_gpu_work(libloc):
    import math
    import paper_1910_00572_gb300 as loc
    import numpy as np
    occ = np.zeros((8, 8), np.uint8)
    for bad in (-0.5, math.nan, math.inf):
        p = loc.loc_params_default(H=8, W=8, K=4, cell_m=0.1, sigma_cross_cells=bad)
        with pytest.raises(loc.LocError) as e:
            loc.loc_create(occ, p)
        assert e.value.status == loc.LOC_ERR_INVALID_ARG
    # the default radius follows the larger sigma: ceil(3 * 1.5) = 5 > LOC_MAX_R_XY
    p = loc.loc_params_default(H=8, W=8, K=4, cell_m=0.1, sigma_xy_cells=0.5, sigma_cross_cells=1.5)
    with pytest.raises(loc.LocError):
        loc.loc_create(occ, p)
    p = loc.loc_params_default(H=8, W=8, K=4, cell_m=0.1, sigma_xy_cells=0.0, sigma_cross_cells=0.5)
    with pytest.raises(loc.LocError):
        loc.loc_create(occ, p)                                  # no sigma along the heading
    p = loc.loc_params_default(H=8, W=8, K=4, cell_m=0.1, sigma_cross_cells=0.8, kernel=loc.LOC_KERNEL_TILED)
    with pytest.raises(loc.LocError) as e:
        loc.loc_create(occ, p)
    assert "generic" in loc.loc_last_error()
    # the allocation-free call takes isotropic noise only; it refuses before touching the pointers
    p = loc.loc_params_default(H=8, W=8, K=4, cell_m=0.1, sigma_cross_cells=0.8)
    with pytest.raises(loc.LocError) as e:
        loc.loc_propagate_noalloc(p, 256, 256, 256, 256, 0.0, 0.0)
    assert e.value.status == loc.LOC_ERR_INVALID_ARG and "anisotropic" in loc.loc_last_error()


def test_huge_or_infinite_sigmas_are_rejected_before_any_conversion(libloc):
    """A default radius ceil(3 sigma) beyond every maximum (or an infinite sigma) is refused
    with INVALID_ARG by the session and the allocation-free call alike, before the pointers
    are touched and without converting an out-of-range double to int."""
    import math
    import paper_1910_00572_gb300 as loc
    import numpy as np
    occ = np.zeros((8, 8), np.uint8)
    for field in ("sigma_xy_cells", "sigma_theta_bins"):
        for bad in (1e12, 1e300, math.inf, 2.0):
            p = loc.loc_params_default(H=8, W=8, K=4, cell_m=0.1, **{field: bad})
            with pytest.raises(loc.LocError) as e:
                loc.loc_create(occ, p)
            assert e.value.status == loc.LOC_ERR_INVALID_ARG
            with pytest.raises(loc.LocError) as e:
                loc.loc_propagate_noalloc(p, 256, 256, 256, 256, 0.0, 0.0)
            assert e.value.status == loc.LOC_ERR_INVALID_ARG
            assert "radius" in loc.loc_last_error() or "finite" in loc.loc_last_error()
