"""Seeded synthetic inputs shared by the CUDA path's tests, the oracle's tests and bench.py.

This package holds none of the filter's arithmetic.  It only *produces inputs*:

* ``floorplan``  -- occupancy maps standing in for the Radish floor plans of the paper's
  evaluation (Section IV), which are not available here: a small rooms-and-doorways plan
  and an office generator (corridors + rooms);
* ``trajectory`` -- a seeded random walk of the ground-truth pose on free space and the
  noisy relative-pose odometry it produces;
* ``scan``       -- a simulated 2-D LIDAR (a brute-force fine ray march from the true
  continuous pose, with range noise and dropouts), standing in for the ISAAC simulator's
  LIDAR (Section IV);
* ``workloads``  -- the named workloads (grid sizes, bins, cell size, noise) used by the
  tests and the benchmark;
* ``fields``     -- seeded random fields (belief-like tensors, belief maps) for stage tests.

Every generator takes an explicit integer seed and uses ``numpy.random.Generator(PCG64)``.
"""
