"""Host logic of bench.py that needs no GPU: the roofline's measured DRAM traffic comes from
the committed ncu summary of the default propagation kernel, and only while the kernel source
is byte-for-byte the one that was captured (its sha256 is in the summary)."""
import os
import sys
from types import SimpleNamespace

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from synth import workloads  # noqa: E402


def test_profile_summary_matches_the_profiled_source():
    """A source change without a fresh capture would silently drop the traffic figure from
    the bench line; this fails first."""
    wl = workloads.get("office512")
    traffic = bench.profiled_traffic(wl, SimpleNamespace(tile=0, kernel=0))
    assert traffic is not None
    alg = wl["H"] * wl["W"] * wl["K"] * 2 * 4 + wl["H"] * wl["W"] * 5
    assert 0.3 * alg < traffic < 1.5 * alg          # DRAM bytes of one launch, near the algorithmic


def test_traffic_is_not_reported_for_other_kernels():
    wl = workloads.get("office512")
    assert bench.profiled_traffic(wl, SimpleNamespace(tile=3, kernel=0)) is None
    assert bench.profiled_traffic(wl, SimpleNamespace(tile=0, kernel=1)) is None
    assert bench.profiled_traffic(workloads.get("office2048"), SimpleNamespace(tile=0, kernel=0)) is None


def test_served_traffic_scales_the_profiled_ratio():
    """The default line's roofline traffic: the batched kernel's profiled DRAM / algorithmic byte
    ratio times the run's algorithmic bytes per launch, tied to the profiled source."""
    t = bench.served_traffic(4.0e10)
    assert t is not None
    assert 0.5 * 4.0e10 < t < 1.5 * 4.0e10
    assert bench.served_traffic(0.0) is None
