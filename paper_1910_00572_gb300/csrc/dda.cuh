// The FP32 grid walk behind the expected range of a state (the likelihood P(z | x) of Eq. 9),
// shared by the sampled scan update (lidar.cu) and the range table of the dense update
// (dense.cu).
#pragma once
#include <cstdint>

namespace loc {

// Distance in cells from the centre of free cell (j, i) along (dx, dy) to the first occupied
// cell or the grid edge, capped at rmax; ties step x first.  Every crossing time is the FP32
// value the reference walk computes, t = fl(fl(n + 1/2) * fl(1 / |d|)), so the decisions and the
// result are the same bit for bit.  free_at(j, i) tells whether an in-grid cell is free.
template <typename FreeAt>
__device__ __forceinline__ float dda_walk(const FreeAt& free_at, int H, int W, int j, int i, float dx, float dy,
                                          float rmax) {
    if (!free_at(j, i)) return 0.0f;
    const int sx = dx > 0.0f ? 1 : -1, sy = dy > 0.0f ? 1 : -1;
    const float tdx = dx != 0.0f ? __fdiv_rn(1.0f, fabsf(dx)) : INFINITY;
    const float tdy = dy != 0.0f ? __fdiv_rn(1.0f, fabsf(dy)) : INFINITY;
    // the next crossings: t_x = (n_x + 1/2) * tdx, t_y likewise, n the cells stepped so far;
    // n + 1/2 is kept as a float (exact: an integer plus one half, far below 2^23) and only the
    // crossing that was taken is recomputed, so every value equals the per-step formula
    float ax = 0.5f, ay = 0.5f;
    float tx = __fmul_rn(ax, tdx), ty = __fmul_rn(ay, tdy);
    // every step crosses one cell boundary and t grows by at least 1/2 cell per two steps
    const int max_steps = 4 * (int)rmax + 16;
    for (int s = 0; s < max_steps; ++s) {
        float t;
        if (tx <= ty) {
            i += sx;
            t = tx;
            ax = __fadd_rn(ax, 1.0f);
            tx = __fmul_rn(ax, tdx);
        } else {
            j += sy;
            t = ty;
            ay = __fadd_rn(ay, 1.0f);
            ty = __fmul_rn(ay, tdy);
        }
        if (t >= rmax) return rmax;
        if ((unsigned)i >= (unsigned)W || (unsigned)j >= (unsigned)H) return t;
        if (!free_at(j, i)) return t;
    }
    return rmax;
}

// The walk on the byte map (1 = free).
__device__ __forceinline__ float dda_cells(const uint8_t* __restrict__ trav, int H, int W, int j, int i, float dx, float dy,
                                           float rmax) {
    return dda_walk([trav, W](int jj, int ii) { return trav[(size_t)jj * W + ii] != 0; }, H, W, j, i, dx, dy, rmax);
}

}  // namespace loc
