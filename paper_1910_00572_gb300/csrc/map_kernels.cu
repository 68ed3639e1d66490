// Create-time and readback kernels: the edge-normalisation field of Eq. 8, the normalised
// belief, the belief map (max or sum over channels, Section III-A.3), the argmax estimate,
// and loading a caller-given belief.
#include <cfloat>
#include <climits>

#include "kernels.h"

namespace loc {
namespace {

constexpr int NT = 256;

// Eq. 8: G(B_0, k) for the binary free-space tensor is the x/y blur of M (the theta taps of
// a theta-constant tensor sum to 1); corr = 1 / G on free cells, 0 on occupied cells.
__global__ void edge_correction_kernel(const uint8_t* __restrict__ trav, float* __restrict__ corr,
                                       int H, int W, const __grid_constant__ StepArgs g) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= W) return;
    const int r = g.r_xy;
    float G = 0.0f;
    for (int dj = -r; dj <= r; ++dj) {
        const int jj = j + dj;
        if (jj < 0 || jj >= H) continue;
        float row = 0.0f;
        for (int di = -r; di <= r; ++di) {
            const int ii = i + di;
            if (ii >= 0 && ii < W) row += g.gx[di + r] * (float)trav[(size_t)jj * W + ii];
        }
        G += g.gx[dj + r] * row;
    }
    const size_t o = (size_t)j * W + i;
    corr[o] = (trav[o] && G > 0.0f) ? 1.0f / G : 0.0f;
}

template <typename T>
__device__ __forceinline__ float belief_at(const T* B, const uint8_t* trav, size_t hw, size_t q,
                                           int reinit, float inv_uniform, float scale) {
    return reinit ? (float)trav[q % hw] * inv_uniform : Store<T>::ld(B + q) * scale;
}

template <typename T>
__global__ void read_belief_kernel(const T* __restrict__ B, const uint8_t* __restrict__ trav,
                                   const SessionDev* sd, float inv_uniform, size_t hw, size_t n,
                                   float* __restrict__ out) {
    const int reinit = sd->reinit;
    const float scale = sd->inv_Z;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (size_t)gridDim.x * blockDim.x)
        out[q] = belief_at(B, trav, hw, q, reinit, inv_uniform, scale);
}

template <typename T>
__global__ void read_marginal_kernel(const T* __restrict__ B, const uint8_t* __restrict__ trav,
                                     const SessionDev* sd, float inv_uniform, size_t hw, int K,
                                     int mode, float* __restrict__ out) {
    const int reinit = sd->reinit;
    const float scale = sd->inv_Z;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < hw;
         q += (size_t)gridDim.x * blockDim.x) {
        float acc = 0.0f;                       // beliefs are non-negative
        for (int k = 0; k < K; ++k) {
            const float v = belief_at(B, trav, hw, (size_t)k * hw + q, reinit, inv_uniform, scale);
            acc = mode == LOC_MAP_MAX ? fmaxf(acc, v) : acc + v;
        }
        out[q] = acc;
    }
}

// (value, index) order: larger value first, then lower index.
__device__ __forceinline__ bool better(float v, long long i, float bv, long long bi) {
    return v > bv || (v == bv && i < bi);
}

template <typename T>
__global__ void argmax_partial_kernel(const T* __restrict__ B, const uint8_t* __restrict__ trav,
                                      const SessionDev* sd, float inv_uniform, size_t hw, size_t n,
                                      float* __restrict__ pv, long long* __restrict__ pi) {
    __shared__ float sv[NT];
    __shared__ long long si[NT];
    const int reinit = sd->reinit;
    float bv = -FLT_MAX;
    long long bi = (long long)n;
    for (size_t q = (size_t)blockIdx.x * NT + threadIdx.x; q < n; q += (size_t)gridDim.x * NT) {
        const float v = belief_at(B, trav, hw, q, reinit, inv_uniform, 1.0f);
        if (better(v, (long long)q, bv, bi)) { bv = v; bi = (long long)q; }
    }
    sv[threadIdx.x] = bv;
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int s = NT / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s && better(sv[threadIdx.x + s], si[threadIdx.x + s], sv[threadIdx.x], si[threadIdx.x])) {
            sv[threadIdx.x] = sv[threadIdx.x + s];
            si[threadIdx.x] = si[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        pv[blockIdx.x] = sv[0];
        pi[blockIdx.x] = si[0];
    }
}

// The same over the stored values with V consecutive elements per 16-byte load (n a multiple
// of V).  Every thread scans its elements in increasing index order, so a strict '>' keeps the
// lowest index among equal values; threads, warps and CTAs combine with better().
// The CTA that finishes last combines the per-CTA results (fixed order, so the result does not
// depend on which CTA is last) and writes the index and the normalised value.
template <typename T, int V>
__global__ void __launch_bounds__(NT) argmax_vec_kernel(const T* __restrict__ B, const uint8_t* __restrict__ trav,
                                                        const SessionDev* sd, float inv_uniform, size_t hw, size_t n,
                                                        float* __restrict__ pv, long long* __restrict__ pi,
                                                        unsigned int* counter, long long* out_idx, float* out_val) {
    static_assert(V * sizeof(T) == 16, "one 16-byte load");
    __shared__ float sv[NT / 32];
    __shared__ long long si[NT / 32];
    float bv = -FLT_MAX;
    long long bi = (long long)n;
    const size_t ng = sd->reinit ? 0 : n / V;
    if (sd->reinit) {                 // the belief reads as uniform over free cells
        for (size_t q = (size_t)blockIdx.x * NT + threadIdx.x; q < n; q += (size_t)gridDim.x * NT) {
            const float v = (float)trav[q % hw] * inv_uniform;
            if (v > bv) {
                bv = v;
                bi = (long long)q;
            }
        }
    }
    for (size_t g = (size_t)blockIdx.x * NT + threadIdx.x; g < ng; g += (size_t)gridDim.x * NT) {
        union {
            uint4 u;
            T x[V];
        } raw;
        raw.u = __ldg(reinterpret_cast<const uint4*>(B) + g);
#pragma unroll
        for (int e = 0; e < V; ++e) {
            const float v = Store<T>::ld(&raw.x[e]);
            if (v > bv) {
                bv = v;
                bi = (long long)(g * V + e);
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_down_sync(0xffffffffu, bv, o);
        const long long oi = __shfl_down_sync(0xffffffffu, bi, o);
        if (better(ov, oi, bv, bi)) {
            bv = ov;
            bi = oi;
        }
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        sv[warp] = bv;
        si[warp] = bi;
    }
    __syncthreads();
    __shared__ int s_last;
    if (threadIdx.x == 0) {
        for (int w = 1; w < NT / 32; ++w)
            if (better(sv[w], si[w], bv, bi)) {
                bv = sv[w];
                bi = si[w];
            }
        pv[blockIdx.x] = bv;
        pi[blockIdx.x] = bi;
        __threadfence();
        s_last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    bv = -FLT_MAX;
    bi = LLONG_MAX;
    for (unsigned int b = threadIdx.x; b < gridDim.x; b += NT) {
        const float v = ((volatile float*)pv)[b];
        const long long q = ((volatile long long*)pi)[b];
        if (better(v, q, bv, bi)) {
            bv = v;
            bi = q;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_down_sync(0xffffffffu, bv, o);
        const long long oi = __shfl_down_sync(0xffffffffu, bi, o);
        if (better(ov, oi, bv, bi)) {
            bv = ov;
            bi = oi;
        }
    }
    __syncthreads();
    if (lane == 0) {
        sv[warp] = bv;
        si[warp] = bi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < NT / 32; ++w)
            if (better(sv[w], si[w], bv, bi)) {
                bv = sv[w];
                bi = si[w];
            }
        *out_idx = bi;
        *out_val = sd->reinit ? bv : (float)((double)bv / sd->Z);
        *counter = 0u;
    }
}

// loc_estimate: one pass over the belief around the argmax state a (written by the argmax
// kernel on the same stream).  mass_near sums the states whose cell lies within the disk
// dj^2 + di^2 <= r2 of a's cell and whose bin is within dk of a's (circular): FP32 Kahan per
// thread, FP64 per CTA, the last CTA summing the CTA partials in a fixed order.  The second
// hypothesis is the largest belief among the cells outside the disk, the lowest cell index on
// ties (threads scan in increasing index order and combine with better()).
template <typename T>
__global__ void __launch_bounds__(NT) estimate_kernel(const T* __restrict__ B, const uint8_t* __restrict__ trav,
                                                      const SessionDev* sd, float inv_uniform, int H, int W, int K,
                                                      const long long* arg_idx, long long r2, int dk,
                                                      double* partials, float* pv, long long* pi,
                                                      unsigned int* counter, EstimateOut* out) {
    __shared__ double red[NT / 32];
    __shared__ float sv[NT / 32];
    __shared__ long long si[NT / 32];
    const size_t hw = (size_t)H * W;
    const long long a = *arg_idx;
    const int ka = (int)(a / (long long)hw), ja = (int)((a % (long long)hw) / W), ia = (int)(a % W);
    const int reinit = sd->reinit;
    const float scale = sd->inv_Z;
    KahanF mass;
    float bv = -FLT_MAX;
    long long bi = LLONG_MAX;
    // one thread per cell (consecutive across a warp), its K bins in turn
    for (size_t cell = (size_t)blockIdx.x * NT + threadIdx.x; cell < hw; cell += (size_t)gridDim.x * NT) {
        const int j = (int)(cell / (unsigned int)W), i = (int)(cell - (size_t)j * W);
        const long long dj = j - ja, di = i - ia;
        const bool inside = dj * dj + di * di <= r2;
        float m = 0.0f;                                   // the cell's belief-map value
#pragma unroll 8
        for (int k = 0; k < K; ++k) {
            const float v = belief_at(B, trav, hw, (size_t)k * hw + cell, reinit, inv_uniform, scale);
            if (inside) {
                int d = k > ka ? k - ka : ka - k;
                if (K - d < d) d = K - d;
                if (d <= dk) mass.add(v);
            } else {
                m = fmaxf(m, v);
            }
        }
        if (!inside && better(m, (long long)cell, bv, bi)) {
            bv = m;
            bi = (long long)cell;
        }
    }
    const double bm = block_sum<NT>(mass.value(), red);
    for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_down_sync(0xffffffffu, bv, o);
        const long long oi = __shfl_down_sync(0xffffffffu, bi, o);
        if (better(ov, oi, bv, bi)) {
            bv = ov;
            bi = oi;
        }
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        sv[warp] = bv;
        si[warp] = bi;
    }
    __syncthreads();
    __shared__ int s_last;
    if (threadIdx.x == 0) {
        for (int w = 1; w < NT / 32; ++w)
            if (better(sv[w], si[w], bv, bi)) {
                bv = sv[w];
                bi = si[w];
            }
        partials[blockIdx.x] = bm;
        pv[blockIdx.x] = bv;
        pi[blockIdx.x] = bi;
        __threadfence();
        s_last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double ms = 0.0;
    bv = -FLT_MAX;
    bi = LLONG_MAX;
    for (unsigned int b = threadIdx.x; b < gridDim.x; b += NT) {
        ms += ((volatile double*)partials)[b];
        const float v = ((volatile float*)pv)[b];
        const long long q = ((volatile long long*)pi)[b];
        if (better(v, q, bv, bi)) {
            bv = v;
            bi = q;
        }
    }
    const double mt = block_sum<NT>(ms, red);
    for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_down_sync(0xffffffffu, bv, o);
        const long long oi = __shfl_down_sync(0xffffffffu, bi, o);
        if (better(ov, oi, bv, bi)) {
            bv = ov;
            bi = oi;
        }
    }
    __syncthreads();
    if (lane == 0) {
        sv[warp] = bv;
        si[warp] = bi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < NT / 32; ++w)
            if (better(sv[w], si[w], bv, bi)) {
                bv = sv[w];
                bi = si[w];
            }
        out->mass_near = mt;
        out->second_p = bv > 0.0f ? bv : 0.0f;
        out->second_cell = bv > 0.0f ? bi : -1;
        *counter = 0u;
    }
}

// The same pass over the flat tensor in 16-byte groups of V consecutive states (hw a multiple
// of V and W >= V, so a group stays in one plane): one division to place a thread's first
// group, then the plane, cell, row and column advance by the grid stride.
template <typename T, int V>
__global__ void __launch_bounds__(NT) estimate_vec_kernel(const T* __restrict__ B, const uint8_t* __restrict__ trav,
                                                          const SessionDev* sd, float inv_uniform, int H, int W,
                                                          int K, const long long* arg_idx, long long r2, int dk,
                                                          double* partials, float* pv, long long* pi,
                                                          unsigned int* counter, EstimateOut* out) {
    static_assert(V * sizeof(T) == 16, "one 16-byte load");
    __shared__ double red[NT / 32];
    __shared__ float sv[NT / 32];
    __shared__ long long si[NT / 32];
    const size_t hw = (size_t)H * W, ng = hw * K / V;
    const long long a = *arg_idx;
    const int ka = (int)(a / (long long)hw), ja = (int)((a % (long long)hw) / W), ia = (int)(a % W);
    const int reinit = sd->reinit;
    const float scale = sd->inv_Z;
    KahanF mass;
    float bv = -FLT_MAX;
    long long bi = LLONG_MAX;
    const size_t g0 = (size_t)blockIdx.x * NT + threadIdx.x, gs = (size_t)gridDim.x * NT;
    if (g0 < ng) {
        size_t q = g0 * V;
        int k = (int)(q / hw);
        size_t cell = q - (size_t)k * hw;
        int j = (int)(cell / (unsigned int)W), i = (int)(cell - (size_t)j * W);
        const size_t step = gs * V;                       // the grid stride in states
        const int dkk = (int)(step / hw);
        const size_t dcell = step - (size_t)dkk * hw;
        const int dj = (int)(dcell / (unsigned int)W), di = (int)(dcell - (size_t)dj * W);
        for (size_t g = g0; g < ng; g += gs) {
            union {
                uint4 u;
                T x[V];
            } raw;
            if (!reinit) raw.u = __ldg(reinterpret_cast<const uint4*>(B) + g);
            int je = j, ie = i;
#pragma unroll
            for (int e = 0; e < V; ++e) {
                if (e > 0 && ++ie == W) {
                    ie = 0;
                    ++je;
                }
                const size_t ce = cell + e;
                const float v = reinit ? (float)trav[ce] * inv_uniform : Store<T>::ld(&raw.x[e]) * scale;
                const long long ddj = je - ja, ddi = ie - ia;
                if (ddj * ddj + ddi * ddi <= r2) {
                    int d = k > ka ? k - ka : ka - k;
                    if (K - d < d) d = K - d;
                    if (d <= dk) mass.add(v);
                } else if (better(v, (long long)ce, bv, bi)) {
                    bv = v;
                    bi = (long long)ce;
                }
            }
            k += dkk;
            cell += dcell;
            j += dj;
            i += di;
            if (i >= W) {
                i -= W;
                ++j;
            }
            if (cell >= hw) {
                cell -= hw;
                j -= H;
                ++k;
            }
        }
    }
    const double bm = block_sum<NT>(mass.value(), red);
    for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_down_sync(0xffffffffu, bv, o);
        const long long oi = __shfl_down_sync(0xffffffffu, bi, o);
        if (better(ov, oi, bv, bi)) {
            bv = ov;
            bi = oi;
        }
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        sv[warp] = bv;
        si[warp] = bi;
    }
    __syncthreads();
    __shared__ int s_last;
    if (threadIdx.x == 0) {
        for (int w = 1; w < NT / 32; ++w)
            if (better(sv[w], si[w], bv, bi)) {
                bv = sv[w];
                bi = si[w];
            }
        partials[blockIdx.x] = bm;
        pv[blockIdx.x] = bv;
        pi[blockIdx.x] = bi;
        __threadfence();
        s_last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double ms = 0.0;
    bv = -FLT_MAX;
    bi = LLONG_MAX;
    for (unsigned int b = threadIdx.x; b < gridDim.x; b += NT) {
        ms += ((volatile double*)partials)[b];
        const float v = ((volatile float*)pv)[b];
        const long long q = ((volatile long long*)pi)[b];
        if (better(v, q, bv, bi)) {
            bv = v;
            bi = q;
        }
    }
    const double mt = block_sum<NT>(ms, red);
    for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_down_sync(0xffffffffu, bv, o);
        const long long oi = __shfl_down_sync(0xffffffffu, bi, o);
        if (better(ov, oi, bv, bi)) {
            bv = ov;
            bi = oi;
        }
    }
    __syncthreads();
    if (lane == 0) {
        sv[warp] = bv;
        si[warp] = bi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < NT / 32; ++w)
            if (better(sv[w], si[w], bv, bi)) {
                bv = sv[w];
                bi = si[w];
            }
        out->mass_near = mt;
        out->second_p = bv > 0.0f ? bv : 0.0f;
        out->second_cell = bv > 0.0f ? bi : -1;
        *counter = 0u;
    }
}

__global__ void argmax_final_kernel(const float* __restrict__ pv, const long long* __restrict__ pi,
                                    int nb, const SessionDev* sd, long long* out_idx,
                                    float* out_val) {
    __shared__ float sv[NT];
    __shared__ long long si[NT];
    float bv = -FLT_MAX;
    long long bi = LLONG_MAX;
    for (int b = threadIdx.x; b < nb; b += NT)
        if (better(pv[b], pi[b], bv, bi)) { bv = pv[b]; bi = pi[b]; }
    sv[threadIdx.x] = bv;
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int s = NT / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s && better(sv[threadIdx.x + s], si[threadIdx.x + s], sv[threadIdx.x], si[threadIdx.x])) {
            sv[threadIdx.x] = sv[threadIdx.x + s];
            si[threadIdx.x] = si[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *out_idx = si[0];
        *out_val = sd->reinit ? sv[0] : (float)((double)sv[0] / sd->Z);
    }
}

template <typename T>
__global__ void set_belief_kernel(const float* __restrict__ src, T* __restrict__ B, size_t n,
                                  float mult, SessionDev* sd, double* partials) {
    __shared__ double red[NT / 32];
    float part = 0.0f;
    double acc = 0.0;
    int cnt = 0;
    for (size_t q = (size_t)blockIdx.x * NT + threadIdx.x; q < n; q += (size_t)gridDim.x * NT) {
        part += Store<T>::st(B + q, src[q] * mult);
        if (++cnt == 64) { acc += (double)part; part = 0.0f; cnt = 0; }
    }
    acc += (double)part;
    const double bt = block_sum<NT>(acc, red);
    finish_sum<NT>(bt, partials, &sd->counter, gridDim.x, red, [sd](double Z) {
        sd->Z = Z;
        sd->inv_Z = (float)(1.0 / Z);
        sd->reinit = 0;
    });
}

constexpr int kArgmaxBlocks = 1024;

// Writes the uniform belief (trav * value) into B when the restart flag is set; the last CTA
// sets Z to its sum and clears the flag.  Every CTA reads the flag before it arrives.
template <typename T>
__global__ void materialize_kernel(T* __restrict__ B, const uint8_t* __restrict__ trav, SessionDev* sd,
                                   float value, size_t hw, int K, double* partials) {
    __shared__ double red[NT / 32];
    if (!sd->reinit) return;                      // uniform over the grid: every CTA agrees
    KahanF acc;
    const size_t n = hw * K;
    for (size_t q = (size_t)blockIdx.x * NT + threadIdx.x; q < n; q += (size_t)gridDim.x * NT)
        acc.add(Store<T>::st(B + q, (float)trav[q % hw] * value));
    const double bt = block_sum<NT>(acc.value(), red);
    finish_sum<NT>(bt, partials, &sd->counter, gridDim.x, red, [sd](double Z) {
        sd->Z = Z;
        sd->inv_Z = (float)(1.0 / Z);
        sd->reinit = 0;
    });
}

}  // namespace

cudaError_t launch_materialize(void* B, int storage, const uint8_t* trav, SessionDev* sd, float value,
                               size_t hw, int K, double* partials, unsigned int nparts, cudaStream_t st) {
    // grid-stride over the tensor with a small grid: almost every call finds the restart flag
    // clear and every CTA returns at once, so the launch should cost little
    unsigned int nb = (unsigned int)((hw * K + NT - 1) / NT);
    if (nb > nparts) nb = nparts;
    if (nb > 304) nb = 304;
    switch (storage) {
        case LOC_F32: materialize_kernel<float><<<nb, NT, 0, st>>>((float*)B, trav, sd, value, hw, K, partials); break;
        case LOC_BF16: materialize_kernel<__nv_bfloat16><<<nb, NT, 0, st>>>((__nv_bfloat16*)B, trav, sd, value, hw, K, partials); break;
        case LOC_F16: materialize_kernel<__half><<<nb, NT, 0, st>>>((__half*)B, trav, sd, value, hw, K, partials); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_edge_correction(const uint8_t* trav, float* corr, int H, int W,
                                   const float* gx, int r, cudaStream_t st) {
    StepArgs g{};
    g.r_xy = r;
    for (int d = 0; d < 2 * r + 1; ++d) g.gx[d] = gx[d];
    dim3 grid((W + NT - 1) / NT, H);
    edge_correction_kernel<<<grid, NT, 0, st>>>(trav, corr, H, W, g);
    return cudaGetLastError();
}

#define LOC_DISPATCH(storage, CALL)                                                   \
    switch (storage) {                                                                \
        case LOC_F32: { using T = float; CALL; } break;                               \
        case LOC_BF16: { using T = __nv_bfloat16; CALL; } break;                      \
        case LOC_F16: { using T = __half; CALL; } break;                              \
        default: return cudaErrorInvalidValue;                                        \
    }

static unsigned int grid_for(size_t n) {
    size_t b = (n + NT - 1) / NT;
    return (unsigned int)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

cudaError_t launch_read_belief(const void* B, int storage, const uint8_t* trav,
                               const SessionDev* sd, float inv_uniform, int H, int W, int K,
                               float* out, cudaStream_t st) {
    const size_t hw = (size_t)H * W, n = hw * K;
    LOC_DISPATCH(storage, (read_belief_kernel<T><<<grid_for(n), NT, 0, st>>>(
                              (const T*)B, trav, sd, inv_uniform, hw, n, out)));
    return cudaGetLastError();
}

cudaError_t launch_read_marginal(const void* B, int storage, const uint8_t* trav,
                                 const SessionDev* sd, float inv_uniform, int H, int W, int K,
                                 int mode, float* out, cudaStream_t st) {
    const size_t hw = (size_t)H * W;
    LOC_DISPATCH(storage, (read_marginal_kernel<T><<<grid_for(hw), NT, 0, st>>>(
                              (const T*)B, trav, sd, inv_uniform, hw, K, mode, out)));
    return cudaGetLastError();
}

size_t argmax_scratch_bytes(size_t) {
    return (size_t)kArgmaxBlocks * (sizeof(float) + sizeof(long long)) + 16;   // + arrival counter
}

cudaError_t launch_argmax(const void* B, int storage, const uint8_t* trav,
                          const SessionDev* sd, float inv_uniform, int H, int W, int K,
                          void* scratch, long long* out_idx, float* out_val, cudaStream_t st) {
    const size_t hw = (size_t)H * W, n = hw * K;
    long long* pi = (long long*)scratch;
    float* pv = (float*)(pi + kArgmaxBlocks);
    unsigned int nb = grid_for(n);
    if (nb > kArgmaxBlocks) nb = kArgmaxBlocks;
    const size_t vec = storage == LOC_F32 ? 4 : 8;
    if (n % vec == 0) {
        // the stored values order the states like the belief (one positive scale)
        nb = grid_for(n / vec);
        if (nb > kArgmaxBlocks) nb = kArgmaxBlocks;
        unsigned int* counter = reinterpret_cast<unsigned int*>(pv + kArgmaxBlocks);
        LOC_DISPATCH(storage, (argmax_vec_kernel<T, 16 / sizeof(T)><<<nb, NT, 0, st>>>(
                                  (const T*)B, trav, sd, inv_uniform, hw, n, pv, pi, counter, out_idx, out_val)));
        return cudaGetLastError();
    } else {
        LOC_DISPATCH(storage, (argmax_partial_kernel<T><<<nb, NT, 0, st>>>(
                                  (const T*)B, trav, sd, inv_uniform, hw, n, pv, pi)));
    }
    argmax_final_kernel<<<1, NT, 0, st>>>(pv, pi, (int)nb, sd, out_idx, out_val);
    return cudaGetLastError();
}

cudaError_t launch_estimate(const void* B, int storage, const uint8_t* trav, const SessionDev* sd,
                            float inv_uniform, int H, int W, int K, void* scratch, const long long* arg_idx,
                            long long r2, int dk, double* partials, unsigned int nparts, EstimateOut* out,
                            cudaStream_t st) {
    const size_t hw = (size_t)H * W;
    long long* pi = (long long*)scratch;
    float* pv = (float*)(pi + kArgmaxBlocks);
    unsigned int* counter = reinterpret_cast<unsigned int*>(pv + kArgmaxBlocks);
    const size_t vec = storage == LOC_F32 ? 4 : 8;
    if (hw % vec == 0 && (size_t)W >= vec) {
        unsigned int nb = grid_for(hw * K / vec);
        if (nb > kArgmaxBlocks) nb = kArgmaxBlocks;
        if (nb > nparts) nb = nparts;
        LOC_DISPATCH(storage, (estimate_vec_kernel<T, 16 / sizeof(T)><<<nb, NT, 0, st>>>(
                                  (const T*)B, trav, sd, inv_uniform, H, W, K, arg_idx, r2, dk, partials, pv, pi,
                                  counter, out)));
        return cudaGetLastError();
    }
    unsigned int nb = grid_for(hw);
    if (nb > kArgmaxBlocks) nb = kArgmaxBlocks;
    if (nb > nparts) nb = nparts;
    LOC_DISPATCH(storage, (estimate_kernel<T><<<nb, NT, 0, st>>>((const T*)B, trav, sd, inv_uniform, H, W, K, arg_idx,
                                                                 r2, dk, partials, pv, pi, counter, out)));
    return cudaGetLastError();
}

cudaError_t launch_set_belief(const float* src, void* B, int storage, size_t n,
                              SessionDev* sd, double* partials, unsigned int nparts,
                              cudaStream_t st) {
    unsigned int nb = grid_for(n);
    if (nb > nparts) nb = nparts;
    LOC_DISPATCH(storage, (set_belief_kernel<T><<<nb, NT, 0, st>>>(src, (T*)B, n, storage_mult(storage),
                                                                    sd, partials)));
    return cudaGetLastError();
}

}  // namespace loc
