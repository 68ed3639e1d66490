// Dense scan update: Eq. 9 on every state from a precomputed expected-range table.
//
// The map is static, so the expected range of every cell along A fixed directions 2 pi a / A
// (A a multiple of K, so bin k's heading is direction k A / K) is cast once with the FP32
// grid walk of the sampled update and stored as an 8-bit code [A][H][W]:
// q = floor(t * inv_step + 0.5) capped at 255, t in cells, each FP32 operation rounded.
// A scan then scores every state: beam b of bin k reads direction (k s + m_b) mod A, s = A/K,
// m_b its offset from the bin heading rounded to the table grid (host), and
//   log L(k, j, i) = -sum_b (z_b - q step)^2 / (2 sigma^2)
// over the used beams; then X <- X exp(log L - c) mult, c = max over states of
// (log L + log X): the most probable state after the update is stored at the storage
// multiplier, so an informative scan (Eq. 9's normaliser far below 1) cannot underflow FP16
// storage.  The new sum becomes the lazy normaliser (Eq. 9's eta).
//
// Kernels:
//  * range_table_kernel: one thread per cell walks all A directions; the writes of one
//    direction are consecutive across a warp.
//  * dense_score_kernel: a CTA of DC = 64 cells stages their table columns in shared memory
//    (16-byte loads, several in flight), regrouped by residue r = a mod s with the first KC - 1
//    rows of each group repeated, so that bins k .. k+KC-1 of a beam are rows DC bytes apart
//    with no wrap; per thread, beams in the outer loop and KC = 32 bins of accumulators in
//    registers.  The code is turned into a
//    float by the 2^23 exponent trick (exact for 0 .. 255) and compared with z_b / step.  It
//    also reads the stored belief for the offset c.
//  * dense_apply_kernel: X exp(log L - c) mult stored with the storage type's rounding, FP32
//    Kahan partial sums per thread, FP64 per CTA, the last CTA combining them in a fixed
//    order.
#include <cfloat>
#include <climits>
#include <type_traits>

#include "dda.cuh"
#include "kernels.h"
#include "tiled_common.cuh"

namespace loc {
namespace {

constexpr int NT = 256;
constexpr int DC = 64;            // cells per score CTA (one per thread)
constexpr int KC = 32;            // bins per register chunk

// Shared bytes of a score CTA's staged table: s residue blocks of K + min(K, KC - 1) rows of DC
// cells (at most 2 A DC).
__host__ __device__ constexpr size_t dense_table_bytes(int A, int K) {
    return ((size_t)(A / K) * (K + (K < KC - 1 ? K : KC - 1)) * DC + 15) / 16 * 16;
}

// Order-preserving map of floats to unsigned ints (for atomicMax on floats).
__device__ __forceinline__ unsigned int f2ord(float f) {
    const unsigned int u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ord2f(unsigned int u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7FFFFFFFu) : ~u);
}

__global__ void __launch_bounds__(NT) range_table_kernel(const uint8_t* __restrict__ trav, int H, int W,
                                                         const float* __restrict__ dirs, int A, float rmax,
                                                         float inv_step, uint8_t* __restrict__ out) {
    const size_t hw = (size_t)H * W;
    for (size_t c = (size_t)blockIdx.x * NT + threadIdx.x; c < hw; c += (size_t)gridDim.x * NT) {
        const int j = (int)(c / W), i = (int)(c % W);
        for (int a = 0; a < A; ++a) {
            const float t = dda_cells(trav, H, W, j, i, dirs[2 * a], dirs[2 * a + 1], rmax);
            const float f = floorf(__fadd_rn(__fmul_rn(t, inv_step), 0.5f));
            out[(size_t)a * hw + c] = (uint8_t)(f > 255.0f ? 255.0f : f);
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(DC) dense_score_kernel(const uint8_t* __restrict__ table,
                                                         const uint8_t* __restrict__ trav, const T* __restrict__ B,
                                                         size_t hw, int K, int A, int s, const int* __restrict__ m,
                                                         const float* __restrict__ zs, int nu, float scale,
                                                         float* __restrict__ logL, unsigned int* maxL) {
    // Us[(r RB + k') DC + t] = code of direction ((k' mod K) s + r) for cell c0 + t, k' < RB =
    // K + min(K, KC - 1): per residue r the K directions r, s + r, ... followed by the first
    // RB - K of them again, so bins k0 .. k0+KC-1 of a beam with m = q s + r sit at rows
    // r RB + ((q + k0) mod K) + 0 .. KC-1, DC bytes apart (compile-time offsets).
    extern __shared__ __align__(16) unsigned char dsm[];
    const int RB = K + (K < KC - 1 ? K : KC - 1);
    uint8_t* Us = dsm;                                            // [s][RB][DC]
    int* sm_r = reinterpret_cast<int*>(dsm + dense_table_bytes(A, K));  // [nu] block row of each beam
    int* sm_q = sm_r + nu;                                        // [nu] its q
    float* sm_z = reinterpret_cast<float*>(sm_q + nu);            // [nu]
    const int t = threadIdx.x;
    const size_t c0 = (size_t)blockIdx.x * DC, c = c0 + t;
    auto put = [&](int a, auto store) {                           // direction a's row(s)
        const int r = a % s, k = a / s;
        store(r * RB + k);
        if (k < RB - K) store(r * RB + K + k);
    };
    if ((hw & 15) == 0 && c0 + DC <= hw) {
        // 16 cells per 16-byte load: DC / 16 threads per direction, 16 directions a pass, four
        // passes in flight
        constexpr int TPD = DC / 16;
        const int g = t % TPD, a0 = t / TPD;
#pragma unroll 4
        for (int a = a0; a < A; a += DC / TPD) {
            const uint4 v = *reinterpret_cast<const uint4*>(table + (size_t)a * hw + c0 + 16 * g);
            put(a, [&](int row) { *reinterpret_cast<uint4*>(Us + (size_t)row * DC + 16 * g) = v; });
        }
    } else {
        for (int a = 0; a < A; ++a) {
            const uint8_t v = c < hw ? table[(size_t)a * hw + c] : (uint8_t)0;
            put(a, [&](int row) { Us[(size_t)row * DC + t] = v; });
        }
    }
    for (int u = t; u < nu; u += DC) {
        sm_r[u] = (m[u] % s) * RB * DC;
        sm_q[u] = m[u] / s;
        sm_z[u] = zs[u];
    }
    __syncthreads();
    const bool in = c < hw, free = in && trav[c] != 0;
    float best = -FLT_MAX;
    for (int k0 = 0; k0 < K; k0 += KC) {
        float acc[KC];
#pragma unroll
        for (int kk = 0; kk < KC; ++kk) acc[kk] = 0.0f;
        // bins k0 .. k0+KC-1 of every used beam (rows stay below r RB + RB).  A full chunk runs
        // bin pairs on the packed FP32 pipe: each lane of a pair is the scalar code's operations
        // on its own bin in the same order, so the sums are the same bit for bit.
        if (k0 + KC <= K) {
            using tiled::f2;
            f2 acc2[KC / 2];
#pragma unroll
            for (int kk = 0; kk < KC / 2; ++kk) acc2[kk] = 0ull;
            const f2 bias = tiled::pk(-8388608.0f, -8388608.0f);
            for (int u = 0; u < nu; ++u) {
                int k1 = sm_q[u] + k0;
                if (k1 >= K) k1 -= K;
                const uint8_t* col = Us + sm_r[u] + k1 * DC + t;
                const f2 zu = tiled::pk(sm_z[u], sm_z[u]);
#pragma unroll
                for (int kk = 0; kk < KC; kk += 2) {
                    const uint32_t q0 = col[kk * DC], q1 = col[(kk + 1) * DC];
                    // the codes as floats (2^23 + q, exact, minus 2^23)
                    const f2 qf = tiled::fadd2(tiled::pk(__uint_as_float(0x4B000000u | q0),
                                                         __uint_as_float(0x4B000000u | q1)), bias);
                    const f2 d = tiled::fsub2(zu, qf);
                    acc2[kk / 2] = tiled::ffma2(d, d, acc2[kk / 2]);
                }
            }
#pragma unroll
            for (int kk = 0; kk < KC; kk += 2) tiled::upk(acc2[kk / 2], acc[kk], acc[kk + 1]);
        } else {
            for (int u = 0; u < nu; ++u) {
                int k1 = sm_q[u] + k0;
                if (k1 >= K) k1 -= K;
                const uint8_t* col = Us + sm_r[u] + k1 * DC + t;
                const float zu = sm_z[u];
#pragma unroll
                for (int kk = 0; kk < KC; ++kk) {
                    if (k0 + kk < K) {
                        const uint32_t q = col[kk * DC];
                        const float qf = __uint_as_float(0x4B000000u | q) - 8388608.0f;
                        const float d = zu - qf;
                        acc[kk] = fmaf(d, d, acc[kk]);
                    }
                }
            }
        }
#pragma unroll
        for (int kk = 0; kk < KC; ++kk) {
            if (k0 + kk < K && in) {
                const size_t q = (size_t)(k0 + kk) * hw + c;
                const float l = free ? -acc[kk] * scale : -INFINITY;
                logL[q] = l;
                const float x = Store<T>::ld(B + q);
                if (free && x > 0.0f) best = fmaxf(best, l + logf(x));
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) best = fmaxf(best, __shfl_down_sync(0xffffffffu, best, o));
    if ((t & 31) == 0 && best > -FLT_MAX) atomicMax(maxL, f2ord(best));
}

template <typename T>
__global__ void __launch_bounds__(NT) dense_apply_kernel(T* __restrict__ B, const float* __restrict__ logL, size_t hw,
                                                         int K, const unsigned int* maxL, float log_mult,
                                                         double* partials, SessionDev* sd) {
    __shared__ double red[NT / 32];
    const float c = ord2f(*maxL);                 // max of log L + log X
    const float off = log_mult - c;
    KahanF acc;
    // one thread per cell, its bins in order: the BF16 rounding residual runs along theta
    for (size_t cell = (size_t)blockIdx.x * NT + threadIdx.x; cell < hw; cell += (size_t)gridDim.x * NT) {
        float res = 0.0f;
        for (int k = 0; k < K; ++k) {
            const size_t q = (size_t)k * hw + cell;
            const float x = Store<T>::ld(B + q);
            // x exp(log L + off) <= mult; for a small x the factor alone could overflow, so a large
            // exponent takes log x in (the multiply keeps x's precision elsewhere)
            const float e = logL[q] + off;
            const float v = x > 0.0f ? (e < 80.0f ? x * expf(e) : expf(e + logf(x))) : 0.0f;
            acc.add(store_diffused<T>(B + q, v, res));
        }
    }
    const double bt = block_sum<NT>(acc.value(), red);
    const unsigned int nblocks = gridDim.x;
    finish_sum<NT>(bt, partials, &sd->counter, nblocks, red, [sd, c, log_mult](double S) {
        const double Z0 = sd->Z;
        if (S > 0.0 && isfinite(S)) {
            // Eq. 9's normaliser: sum(b exp(log L)) = S exp(c) / (mult Z0)
            sd->Z = S;
            sd->inv_Z = (float)(1.0 / S);
            sd->logscale += log(S) - log(Z0) + (double)c - (double)log_mult;
        } else {
            if (!isfinite(S)) sd->status |= LOC_DEV_ERR_NONFINITE_Z;
            sd->Z = 1.0;
            sd->inv_Z = 1.0f;
            sd->reinit = 1;
            sd->n_reinit += 1;
        }
    });
}

// Probe columns for the map difficulty: out[p A + a] = table[a][probes[p]], flag[p] = M there.
__global__ void __launch_bounds__(NT) gather_columns_kernel(const uint8_t* __restrict__ table,
                                                            const uint8_t* __restrict__ trav, size_t hw, int A,
                                                            const int32_t* __restrict__ probes, int n,
                                                            uint8_t* __restrict__ out, uint8_t* __restrict__ flag) {
    const size_t total = (size_t)n * A;
    for (size_t q = (size_t)blockIdx.x * NT + threadIdx.x; q < total; q += (size_t)gridDim.x * NT) {
        const int p = (int)(q / A), a = (int)(q % A);
        out[q] = table[(size_t)a * hw + probes[p]];
        if (a == 0) flag[p] = trav[probes[p]];
    }
}

__device__ __forceinline__ bool better_f(float v, long long i, float bv, long long bi) {
    return v > bv || (v == bv && i < bi);
}

// argmax of a float array (the first index among equal values): per-thread scans in
// increasing index order, warps and CTAs combined with better_f, the last CTA combining the
// CTA results in a fixed order and writing the index to *out.
__global__ void __launch_bounds__(NT) argmax_f32_kernel(const float* __restrict__ x, size_t n, float* pv,
                                                        long long* pi, unsigned int* counter, long long* out) {
    __shared__ float sv[NT / 32];
    __shared__ long long si[NT / 32];
    __shared__ int s_last;
    float bv = -INFINITY;
    long long bi = LLONG_MAX;
    for (size_t q = (size_t)blockIdx.x * NT + threadIdx.x; q < n; q += (size_t)gridDim.x * NT) {
        const float v = x[q];
        if (better_f(v, (long long)q, bv, bi)) {
            bv = v;
            bi = (long long)q;
        }
    }
    auto reduce = [&]() {
        for (int o = 16; o > 0; o >>= 1) {
            const float ov = __shfl_down_sync(0xffffffffu, bv, o);
            const long long oi = __shfl_down_sync(0xffffffffu, bi, o);
            if (better_f(ov, oi, bv, bi)) {
                bv = ov;
                bi = oi;
            }
        }
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        __syncthreads();
        if (lane == 0) {
            sv[warp] = bv;
            si[warp] = bi;
        }
        __syncthreads();
        if (threadIdx.x == 0)
            for (int w = 1; w < NT / 32; ++w)
                if (better_f(sv[w], si[w], bv, bi)) {
                    bv = sv[w];
                    bi = si[w];
                }
    };
    reduce();
    if (threadIdx.x == 0) {
        pv[blockIdx.x] = bv;
        pi[blockIdx.x] = bi;
        __threadfence();
        s_last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    bv = -INFINITY;
    bi = LLONG_MAX;
    for (unsigned int b = threadIdx.x; b < gridDim.x; b += NT) {
        const float v = ((volatile float*)pv)[b];
        const long long q = ((volatile long long*)pi)[b];
        if (better_f(v, q, bv, bi)) {
            bv = v;
            bi = q;
        }
    }
    reduce();
    if (threadIdx.x == 0) {
        *out = bi;
        *counter = 0u;
    }
}

}  // namespace

constexpr unsigned int kArgmaxF32Blocks = 512;

size_t argmax_f32_scratch_bytes() { return (size_t)kArgmaxF32Blocks * (sizeof(float) + sizeof(long long)) + 16; }

cudaError_t launch_gather_columns(const uint8_t* table, const uint8_t* trav, int H, int W, int A,
                                  const int32_t* probes, int n, uint8_t* out, uint8_t* flag, cudaStream_t st) {
    const size_t total = (size_t)n * A;
    size_t nb = (total + NT - 1) / NT;
    if (nb > 4096) nb = 4096;
    if (nb < 1) nb = 1;
    gather_columns_kernel<<<(unsigned int)nb, NT, 0, st>>>(table, trav, (size_t)H * W, A, probes, n, out, flag);
    return cudaGetLastError();
}

cudaError_t launch_argmax_f32(const float* x, size_t n, void* scratch, long long* out, cudaStream_t st) {
    long long* pi = (long long*)scratch;
    float* pv = (float*)(pi + kArgmaxF32Blocks);
    unsigned int* counter = reinterpret_cast<unsigned int*>(pv + kArgmaxF32Blocks);
    size_t nb = (n + NT - 1) / NT;
    if (nb > kArgmaxF32Blocks) nb = kArgmaxF32Blocks;
    if (nb < 1) nb = 1;
    argmax_f32_kernel<<<(unsigned int)nb, NT, 0, st>>>(x, n, pv, pi, counter, out);
    return cudaGetLastError();
}

size_t dense_score_smem(int A, int K, int nu) { return dense_table_bytes(A, K) + (size_t)nu * 12; }

cudaError_t launch_range_table(const uint8_t* trav, int H, int W, const float* dirs, int A, float rmax,
                               float inv_step, uint8_t* out, cudaStream_t st) {
    const size_t hw = (size_t)H * W;
    size_t nb = (hw + NT - 1) / NT;
    if (nb > 65535) nb = 65535;
    range_table_kernel<<<(unsigned int)nb, NT, 0, st>>>(trav, H, W, dirs, A, rmax, inv_step, out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t score_t(const uint8_t* table, const uint8_t* trav, const void* B, int H, int W, int K, int A,
                    const int* m, const float* zs, int nu, float scale, float* logL, unsigned int* maxL,
                    cudaStream_t st) {
    const size_t hw = (size_t)H * W;
    const size_t smem = dense_score_smem(A, K, nu);
    static size_t attr[64] = {};                   // per device: the largest size set so far
    int dev = 0;
    cudaGetDevice(&dev);
    if (smem > 48 * 1024 && (dev < 0 || dev >= 64 || smem > attr[dev])) {
        const cudaError_t e = cudaFuncSetAttribute(dense_score_kernel<T>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) attr[dev] = smem;
    }
    const unsigned int nb = (unsigned int)((hw + DC - 1) / DC);
    dense_score_kernel<T><<<nb, DC, smem, st>>>(table, trav, static_cast<const T*>(B), hw, K, A, A / K, m, zs, nu,
                                                scale, logL, maxL);
    return cudaGetLastError();
}

cudaError_t launch_dense_score(const uint8_t* table, const uint8_t* trav, const void* B, int storage, int H, int W,
                               int K, int A, const int* m, const float* zs, int nu, float scale, float* logL,
                               unsigned int* maxL, cudaStream_t st) {
    if (A % K != 0) return cudaErrorInvalidValue;
    switch (storage) {
        case LOC_F32: return score_t<float>(table, trav, B, H, W, K, A, m, zs, nu, scale, logL, maxL, st);
        case LOC_BF16: return score_t<__nv_bfloat16>(table, trav, B, H, W, K, A, m, zs, nu, scale, logL, maxL, st);
        case LOC_F16: return score_t<__half>(table, trav, B, H, W, K, A, m, zs, nu, scale, logL, maxL, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_dense_apply(void* B, int storage, const float* logL, size_t hw, int K, const unsigned int* maxL,
                               float log_mult, double* partials, unsigned int nparts, SessionDev* sd,
                               cudaStream_t st) {
    size_t nb = (hw + NT - 1) / NT;
    if (nb > nparts) nb = nparts;
    if (nb > 4096) nb = 4096;
    if (nb < 1) nb = 1;
    switch (storage) {
        case LOC_F32:
            dense_apply_kernel<float><<<(unsigned int)nb, NT, 0, st>>>((float*)B, logL, hw, K, maxL, log_mult, partials, sd);
            break;
        case LOC_BF16:
            dense_apply_kernel<__nv_bfloat16><<<(unsigned int)nb, NT, 0, st>>>((__nv_bfloat16*)B, logL, hw, K, maxL,
                                                                               log_mult, partials, sd);
            break;
        case LOC_F16:
            dense_apply_kernel<__half><<<(unsigned int)nb, NT, 0, st>>>((__half*)B, logL, hw, K, maxL, log_mult, partials, sd);
            break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace loc
