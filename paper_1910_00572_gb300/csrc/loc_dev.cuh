// Device-side definitions shared by the localizer's kernels (not by any test helper).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "loc.h"

namespace loc {

// Source offset of the bilinear pull of Eq. 3 for one channel: output (j, i) reads
// (j + oy + {0,1}, i + ox + {0,1}) with weights (1-fy|fy) x (1-fx|fx).
struct Shift {
    int ox, oy;
    float fx, fy;
};

// Device-resident scalars of one session.  The stored tensor X is unnormalised: the
// belief is X / Z.  `reinit` marks X as invalid, to be read as uniform over free cells
// (after Z == 0, and right after creation).
struct SessionDev {
    double Z;                      // sum of the stored tensor (the Eq. 9 normaliser)
    double logscale;               // running sum of log Z over propagations
    unsigned int counter;          // last-block-done counter of the reducing kernels
    int reinit;                    // 1: read the stored tensor as uniform over free cells
    int status;                    // device error bits (LOC_DEV_ERR_*)
    int pad;
    unsigned long long n_reinit;   // restarts after Z == 0
    unsigned long long n_prop;     // propagations done on the device
    float inv_Z;                   // (float)(1 / Z), written with Z (one FP64 division per step)
    int pad2;
};

// Compensated (Kahan) FP32 running sum: a thread's share of the normaliser stays in FP32
// registers (FP64 arithmetic is slow on this GPU) with an error of a few FP32 ulps of the
// total, and is widened to FP64 once for the FP64 block and grid reduction.
struct KahanF {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float x) {
        const float y = x - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

enum { LOC_DEV_ERR_NONFINITE_Z = 1, LOC_DEV_ERR_TIMEOUT = 2 };

// Arguments of one propagation (Algorithm 1's propagation + the Eq. 9 sum) for one session.
struct StepArgs {
    const void* B_in;              // stored tensor X_{t-1}, [K][H][W] of the storage type
    void* B_out;                   // X_t
    const uint8_t* trav;           // M: 1 free, 0 occupied, [H][W]
    const float* corr;             // G(B_0)^-1 on free cells, 0 on occupied, [H][W]
    SessionDev* sd;
    double* partials;              // one FP64 partial sum per CTA
    // the fused argmax of the tiled kernels: per-CTA candidates (value, index) and the result
    // (index of X_t's largest stored value, lowest on ties, or -1; its normalised belief)
    float* am_pv;
    long long* am_pi;
    long long* am_idx;
    float* am_val;
    float inv_uniform;             // 1 / (K * n_free): the uniform belief value
    float out_mult;                // storage multiplier of the outputs (FP16: 2^14, else 1)
    double log_out_mult;           // log(out_mult), removed from the log-scale
    int H, W, K;
    int r_xy, r_th;
    float gx[2 * LOC_MAX_R_XY + 1];     // x and y taps (isotropic), normalised
    float gt[2 * LOC_MAX_R_THETA + 1];  // theta taps, normalised
    // anisotropic motion noise (step_aniso.cu only): channel k's heading is phi0 + dphi * k,
    // sigma_a along it and sigma_c across it (cells)
    float phi0, dphi, sigma_a, sigma_c;
    Shift sh[LOC_MAX_K];
};

// Storage multiplier: FP16 keeps the belief scaled by 2^14 so that values of ~1e-9 stay
// representable while the largest possible value (a normalised 1 times the edge correction,
// below 2) stays far below 65504.  FP32 and BF16 have the FP32 exponent range: 1.
inline float storage_mult(int storage) { return storage == LOC_F16 ? 16384.0f : 1.0f; }

// BF16 by error diffusion along theta, for the propagation kernels: each cell carries a residual
// r from one output plane to the next.  The stored value is the BF16 neighbour of v (the largest
// BF16 value <= v, or the next one above it) nearest to v + r, and r becomes (v + r) - stored.
// So every stored value is within one BF16 unit in the last place of v, and a cell's states keep
// their total mass to within the last residual: rounding does not random-walk the mass of a
// concentrated hypothesis from step to step, as independent per-value rounding does.
__device__ __forceinline__ __nv_bfloat16 bf16_diffuse(float v, float& r) {
    const float w = v + r;
    const int rn = (short)__bfloat16_as_ushort(__float2bfloat16_rn(w));   // negative w: below 0
    const int lo = (int)(__float_as_uint(v) >> 16);
    const int d = min(max(rn, lo), lo + 1);
    r = w - __uint_as_float((uint32_t)d << 16);
    return __ushort_as_bfloat16((unsigned short)d);
}

// Store one propagated value of a cell whose BF16 residual is r: FP32 as is, BF16 by error
// diffusion, FP16 round-to-nearest.  Returns the stored value as FP32.
template <typename T> __device__ __forceinline__ float store_diffused(T* p, float v, float& r);
template <> __device__ __forceinline__ float store_diffused<float>(float* p, float v, float&) {
    *p = v;
    return v;
}
template <> __device__ __forceinline__ float store_diffused<__nv_bfloat16>(__nv_bfloat16* p, float v, float& r) {
    const __nv_bfloat16 b = bf16_diffuse(v, r);
    *p = b;
    return __bfloat162float(b);
}
template <> __device__ __forceinline__ float store_diffused<__half>(__half* p, float v, float&) {
    const __half b = __float2half_rn(v);
    *p = b;
    return __half2float(b);
}

template <typename T> struct Store;
template <> struct Store<float> {
    static __device__ __forceinline__ float ld(const float* p) { return *p; }
    static __device__ __forceinline__ float st(float* p, float v) { *p = v; return v; }
};
template <> struct Store<__nv_bfloat16> {
    static __device__ __forceinline__ float ld(const __nv_bfloat16* p) { return __bfloat162float(*p); }
    static __device__ __forceinline__ float st(__nv_bfloat16* p, float v) {
        __nv_bfloat16 b = __float2bfloat16_rn(v);
        *p = b;
        return __bfloat162float(b);
    }
};
template <> struct Store<__half> {
    static __device__ __forceinline__ float ld(const __half* p) { return __half2float(*p); }
    static __device__ __forceinline__ float st(__half* p, float v) {
        __half b = __float2half_rn(v);
        *p = b;
        return __half2float(b);
    }
};

// Deterministic FP64 block sum of one value per thread (fixed shuffle tree, fixed warp
// order); the result is valid in thread 0.
template <int NT>
__device__ __forceinline__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0) {
        for (int w = 0; w < NT / 32; ++w) s += red[w];
    }
    __syncthreads();
    return s;
}

// Last-block-done finish of a reduction: every CTA stores its partial; the CTA that
// arrives last sums all partials in a fixed order (strided per thread, then the fixed
// block tree), so the result does not depend on which CTA is last, and calls
// `fin(total)` from thread 0.  `red` needs NT/32 doubles.
template <int NT, typename Fin>
__device__ __forceinline__ void finish_sum(double block_total, double* partials,
                                           unsigned int* counter, unsigned int nblocks,
                                           double* red, Fin fin) {
    __shared__ int s_last;
    if (threadIdx.x == 0) {
        partials[blockIdx.x + gridDim.x * blockIdx.y] = block_total;
        __threadfence();
        unsigned int prev = atomicAdd(counter, 1u);
        s_last = (prev == nblocks - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double s = 0.0;
    for (unsigned int b = threadIdx.x; b < nblocks; b += NT)
        s += ((volatile double*)partials)[b];
    double tot = block_sum<NT>(s, red);
    if (threadIdx.x == 0) {
        *counter = 0u;
        fin(tot);
    }
}

}  // namespace loc
