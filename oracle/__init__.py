"""CPU oracle for map-corrected odometry localization (Peng & Weikersdorfer, arXiv 1910.00572).

TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.  Only ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py`` (its CPU-baseline leg and its ``--impl reference`` arm) may import, call,
link or run anything in this package.  The CUDA library never imports it, and this package
never imports the CUDA library: the two share no code.

What is here, each function citing the passage it follows:

* ``odometry``  Section III-A (theta_t = theta_{t-1} + w), Eq. 2 (per-channel motion),
                Alg. 1 (the |u_{t,k}| >= 1 gate) -- FP64.
* ``filter``    Eq. 3 (AF shift, bilinear), Algorithm 1's propagation (mask, 3-D Gaussian blur of
                Eq. 5-7, mask, edge normalisation of Eq. 8), the normaliser eta of Eq. 9 --
                FP64, direct sums (the 3-D convolution is the plain triple sum with the joint
                kernel exp(-1/2 d^T Sigma^-1 d), not a separable pass).
* ``cprop``     the propagation of ``filter`` restated in plain C (``prop.c``): the same
                direct sums in the same order, bit-identical, with the channels spread over
                OpenMP threads, for long trajectories and the all-cores CPU baseline.
* ``aniso``     Eq. 5-6 with sigma_x != sigma_y: the motion kernel rotated to each output
                channel's heading, the per-channel 3-D convolution and edge correction --
                FP64, direct sums.
* ``readout``   belief map (max over channels) and the estimate (its argmax), Section III-A.3.
* ``lidar``     Section III-B: Floyd-Steinberg sample selection (III-B.1), the expected range
                of a state by grid ray casting, the Gaussian range likelihood and the Eq. 9
                reweighting of the sampled states.  FS and the ray cast decide integers
                (selected or not, which cell is hit), so they run in FP32 with a fixed
                operation order (plain C, ``ref.c``, built with contraction off); scoring and
                reweighting are FP64.

Every function here is pinned by ``tests/test_oracle_*.py`` to something other than itself:
closed forms, invariants (mass conservation, exact permutations, zero mass on occupied
cells), brute force on tiny grids (the explicit transition matrix of Eq. 4), analytic wall
distances, and hand-worked dithering examples.
"""
