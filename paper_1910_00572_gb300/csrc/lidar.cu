// LIDAR sample update of Section III-B: belief map -> Floyd-Steinberg sample selection
// (III-B.1) -> expected ranges by grid ray casting -> Gaussian range likelihood -> Eq. 9 on
// the sampled states (the sampled set keeps its mass).
//
// The two steps whose results are integers decided by floating point -- the dithering and
// the ray walk -- use FP32 with every operation explicitly rounded (__fadd_rn / __fmul_rn /
// __fdiv_rn, so nothing is contracted into an FMA) in a fixed order.
#include <algorithm>
#include <cfloat>

#include "dda.cuh"
#include "kernels.h"

namespace loc {
namespace {

constexpr int NT = 256;
constexpr unsigned long long kSpinNs = 200ull * 1000 * 1000;

// Limit of the bounded waits of the Floyd-Steinberg block hand-offs, and the test hook that
// makes them wait on a flag nothing sets (so that the limit runs out and the kernel returns
// with LOC_DEV_ERR_TIMEOUT).  Set by set_fs_wait (loc_debug_fs_stall).
__device__ unsigned long long g_fs_wait_ns = kSpinNs;
__device__ int g_fs_stall = 0;

__device__ __forceinline__ unsigned long long gtime() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ------------------------------------------------------------------ belief map and fs

// m[q] = max_k belief(k, q) (normalised, FP32); the last CTA writes fs = n_samples / sum(m)
// (FP64 sum, rounded to FP32), or 0 when the map is empty.
template <typename T>
__global__ void __launch_bounds__(NT) belief_map_kernel(const T* __restrict__ B, const uint8_t* __restrict__ trav,
                                                        SessionDev* sd, float inv_uniform, size_t hw, int K,
                                                        float* __restrict__ m, double* partials,
                                                        unsigned int* counter, int n_samples, float* fs_out) {
    __shared__ double red[NT / 32];
    const int reinit = sd->reinit;
    const float scale = sd->inv_Z;
    KahanF acc;
    for (size_t q = (size_t)blockIdx.x * NT + threadIdx.x; q < hw; q += (size_t)gridDim.x * NT) {
        float v = 0.0f;
        if (reinit) {
            v = (float)trav[q] * inv_uniform;
        } else {
            for (int k = 0; k < K; ++k) v = fmaxf(v, Store<T>::ld(B + (size_t)k * hw + q) * scale);
        }
        m[q] = v;
        acc.add(v);
    }
    const double bt = block_sum<NT>(acc.value(), red);
    finish_sum<NT>(bt, partials, counter, gridDim.x, red, [fs_out, n_samples](double S) {
        *fs_out = S > 0.0 ? (float)((double)n_samples / S) : 0.0f;
    });
}

// The same with V consecutive cells per thread and 16-byte loads (hw a multiple of V).
template <typename T, int V>
__global__ void __launch_bounds__(NT) belief_map_vec_kernel(const T* __restrict__ B, const uint8_t* __restrict__ trav,
                                                            SessionDev* sd, float inv_uniform, size_t hw, int K,
                                                            float* __restrict__ m, double* partials,
                                                            unsigned int* counter, int n_samples, float* fs_out) {
    static_assert(V * sizeof(T) == 16, "one 16-byte load per plane");
    __shared__ double red[NT / 32];
    const int reinit = sd->reinit;
    const float scale = sd->inv_Z;
    KahanF acc;
    const size_t ng = hw / V;
    for (size_t g = (size_t)blockIdx.x * NT + threadIdx.x; g < ng; g += (size_t)gridDim.x * NT) {
        float v[V];
#pragma unroll
        for (int e = 0; e < V; ++e) v[e] = 0.0f;
        if (reinit) {
#pragma unroll
            for (int e = 0; e < V; ++e) v[e] = (float)trav[g * V + e] * inv_uniform;
        } else {
            for (int k = 0; k < K; ++k) {
                union {
                    uint4 u;
                    T x[V];
                } raw;
                raw.u = __ldg(reinterpret_cast<const uint4*>(B + (size_t)k * hw) + g);
#pragma unroll
                for (int e = 0; e < V; ++e) v[e] = fmaxf(v[e], Store<T>::ld(&raw.x[e]) * scale);
            }
        }
#pragma unroll
        for (int e = 0; e < V; e += 4)
            *reinterpret_cast<float4*>(m + g * V + e) = make_float4(v[e], v[e + 1], v[e + 2], v[e + 3]);
#pragma unroll
        for (int e = 0; e < V; ++e) acc.add(v[e]);
    }
    const double bt = block_sum<NT>(acc.value(), red);
    finish_sum<NT>(bt, partials, counter, gridDim.x, red, [fs_out, n_samples](double S) {
        *fs_out = S > 0.0 ? (float)((double)n_samples / S) : 0.0f;
    });
}

// ------------------------------------------------------------------ Floyd-Steinberg

// One CTA of kFsWarps warps.  Warp w takes the 32-row blocks rb = w, w + kFsWarps, ...; lane l
// owns row 32 rb + l and handles column i = t - 2l at step t, so the three errors it needs from
// the row above (columns i-1, i, i+1) were produced by lane l-1 at steps t-3, t-2, t-1 and
// arrive by warp shuffle.  Lane 0 takes the row above from the previous block's last row,
// which that block's lane 31 writes into bnd[rb][*] and publishes in prog[rb] (columns
// written); every wait on prog is bounded.
//
// Each warp keeps a ring of three 32-column chunks per row in shared memory (column i at
// position i mod 96).  A lane reads min(1, m fs) of its cell there and writes its selection
// back in its place.  Steps run in windows of 32: at step 32 T the last lane has finished chunk
// T - 3 (at step 32 T - 3), so the warp copies that chunk's selections to sel (each lane its own
// row) and stores chunk T of the map (loaded into registers, coalesced, one window earlier) in
// its place.  Terms of the error sum whose source lies outside the grid are zero (their errors
// were never produced), so the sum always takes the same four terms in the same order; only
// the right neighbour above is masked at the last column.
constexpr size_t kScoreWindowBytes = 96 * 1024;   // shared memory for the score kernel's map window
constexpr int kScoreNT = 384;                      // score kernel threads: 360 beam directions in one round
constexpr int kFsWarps = 16;
constexpr int kFsPitch = 97;              // 3 x 32 columns + 1: lane accesses hit distinct banks

__global__ void __launch_bounds__(kFsWarps * 32) fs_kernel(const float* __restrict__ m, const float* fs_ptr, int H,
                                                           int W, uint8_t* __restrict__ sel, int* __restrict__ rowcnt,
                                                           float* bnd, int* prog, int* status) {
    extern __shared__ float fs_ring_all[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float* ring = fs_ring_all + (size_t)warp * 32 * kFsPitch;
    float* own = ring + lane * kFsPitch;                       // this lane's row
    const float fs = *fs_ptr;
    const unsigned long long wait_ns = g_fs_wait_ns;
    const int stall = g_fs_stall;
    const int nrb = (H + 31) / 32, nch = (W + 31) / 32;
    const int vec = (W & 3) == 0 ? 4 : 1;
    const float w7 = 0.4375f, w3 = 0.1875f, w5 = 0.3125f, w1 = 0.0625f;
    for (int rb = warp; rb < nrb; rb += kFsWarps) {
        const int j0 = 32 * rb, j = j0 + lane;
        const bool row_ok = j < H;
        float pre[32];                                         // column 32 c + lane of rows j0 ..
        const bool interior = j0 + 31 < H;                     // every row of the block in the grid
        auto load_chunk = [&](int c) {
            const int col = 32 * c + lane;
            if (interior && col < W) {
                const float* src = m + (size_t)j0 * W + col;
#pragma unroll
                for (int r = 0; r < 32; ++r) pre[r] = src[(size_t)r * W];
            } else {
#pragma unroll
                for (int r = 0; r < 32; ++r)
                    pre[r] = (j0 + r < H && col < W) ? m[(size_t)(j0 + r) * W + col] : 0.0f;
            }
        };
        auto store_chunk = [&](int c) {
            float* dst = ring + (c % 3) * 32 + lane;
#pragma unroll
            for (int r = 0; r < 32; ++r) {
                float v = __fmul_rn(pre[r], fs);
                if (v > 1.0f) v = 1.0f;
                dst[r * kFsPitch] = v;
            }
        };
        int cnt = 0;
        auto copy_out = [&](int c) {                           // this lane's selections of chunk c
            const float* src = own + (c % 3) * 32;
            const int c0 = 32 * c, n = min(32, W - c0);
            uint8_t* out = sel + (size_t)j * W + c0;
            if (!row_ok) return;
            if (vec == 4) {
                for (int k = 0; k < n; k += 4) {
                    const uint32_t b = (uint32_t)__float_as_uint(src[k]) | ((uint32_t)__float_as_uint(src[k + 1]) << 8) |
                                       ((uint32_t)__float_as_uint(src[k + 2]) << 16) |
                                       ((uint32_t)__float_as_uint(src[k + 3]) << 24);
                    *reinterpret_cast<uint32_t*>(out + k) = b;
                    cnt += __popc(b);
                }
            } else {
                for (int k = 0; k < n; ++k) {
                    const uint32_t b = __float_as_uint(src[k]);
                    out[k] = (uint8_t)b;
                    cnt += (int)b;
                }
            }
        };
        __syncwarp();                                          // the previous block's reads are done
        load_chunk(0);
        store_chunk(0);
        if (nch > 1) load_chunk(1);
        __syncwarp();
        float up_old = 0.0f, up_mid = 0.0f, up_new = 0.0f;   // row above: columns i-1, i, i+1
        float e_prev = 0.0f, last = 0.0f;                      // own error at i-1; newest error
        float chunk = 0.0f;                                    // lane L: bnd[rb][t0 + 1 + L]
        bool failed = false;
        const bool publish = lane == 31 && rb + 1 < nrb;       // the next block reads this row
        float* bnd_next = publish ? bnd + (size_t)(rb + 1) * W : bnd;
        const int steps = W + 62;
        const int nwin = (steps + 31) / 32;
        int ri = (96 - 2 * lane) % 96;                         // (t - 2 lane) mod 96
        for (int T = 0; T < nwin; ++T) {
            const int t0 = 32 * T;
            if (rb > 0) {
                // the row above for columns t0+1 .. t0+32 must be published before lane 0 uses it
                const int need = min(W, t0 + 33);
                int ok = 1;
                if (lane == 0) {
                    const unsigned long long g0 = gtime();
                    unsigned int it = 0;
                    while (stall || ((volatile int*)prog)[rb] < need) {
                        if (++it > (1u << 26) || gtime() - g0 > wait_ns) {
                            ok = 0;
                            break;
                        }
                    }
                }
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (!ok) {
                    failed = true;
                    if (lane == 0) atomicOr(status, LOC_DEV_ERR_TIMEOUT);
                    break;
                }
                __threadfence_block();
                const int c = t0 + 1 + lane;
                chunk = c < W ? ((volatile float*)bnd)[(size_t)rb * W + c] : 0.0f;
                // lane 0 starts at column 0 at once: the row above at column 0 must already be
                // in its register chain (other lanes shift theirs in while they wait to start)
                if (T == 0 && lane == 0) up_new = ((volatile float*)bnd)[(size_t)rb * W];
            }
            if (T >= 3 && T - 3 < nch) copy_out(T - 3);
            if (T > 0 && T < nch) {
                __syncwarp();                                  // chunk T - 3 is read and copied
                store_chunk(T);
                __syncwarp();
                if (T + 1 < nch) load_chunk(T + 1);
            }
            if (interior && t0 >= 62 && t0 + 31 <= W - 2) {
                // Every lane's column lies in [0, W - 2] for the whole window and every row of the
                // block is in the grid: no column or row guards, the right neighbour above always
                // exists, and lane 31 publishes its progress once, after the window.  The same
                // operations in the same order as the general steps below (0 + x == x exactly,
                // and chunk is 0 when there is no row above).
#pragma unroll
                for (int s = 0; s < 32; ++s) {
                    const float from_above = __shfl_sync(0xffffffffu, chunk, s);
                    const float from_left = __shfl_up_sync(0xffffffffu, last, 1);
                    up_old = up_mid;
                    up_mid = up_new;
                    up_new = lane == 0 ? from_above : from_left;
                    const float v = own[ri];
                    float E = __fmul_rn(up_old, w1);
                    E = __fadd_rn(E, __fmul_rn(up_mid, w5));
                    E = __fadd_rn(E, __fmul_rn(up_new, w3));
                    E = __fadd_rn(E, __fmul_rn(e_prev, w7));
                    const float val = __fadd_rn(v, E);
                    const bool on = val >= 0.5f;
                    const float err = on ? __fsub_rn(val, 1.0f) : val;
                    own[ri] = __uint_as_float(on ? 1u : 0u);
                    e_prev = err;
                    last = err;
                    if (publish) bnd_next[t0 + s - 62] = err;
                    ri = ri == 95 ? 0 : ri + 1;
                }
                if (publish) {
                    __threadfence_block();
                    ((volatile int*)prog)[rb + 1] = t0 - 30;      // columns 0 .. t0 - 31 written
                }
                continue;
            }
#pragma unroll
            for (int s = 0; s < 32; ++s) {
                const float from_above = __shfl_sync(0xffffffffu, chunk, s);
                const float from_left = __shfl_up_sync(0xffffffffu, last, 1);
                const float incoming = lane == 0 ? (rb > 0 ? from_above : 0.0f) : from_left;
                up_old = up_mid;
                up_mid = up_new;
                up_new = incoming;
                const int i = t0 + s - 2 * lane;
                const float v = own[ri];
                if ((unsigned)i < (unsigned)W && row_ok) {
                    float E = __fadd_rn(0.0f, __fmul_rn(up_old, w1));
                    E = __fadd_rn(E, __fmul_rn(up_mid, w5));
                    E = __fadd_rn(E, __fmul_rn(i + 1 < W ? up_new : 0.0f, w3));
                    E = __fadd_rn(E, __fmul_rn(e_prev, w7));
                    const float val = __fadd_rn(v, E);
                    const bool on = val >= 0.5f;
                    const float err = on ? __fsub_rn(val, 1.0f) : val;
                    own[ri] = __uint_as_float(on ? 1u : 0u);
                    e_prev = err;
                    last = err;
                    if (lane == 31 && rb + 1 < nrb) {
                        bnd[(size_t)(rb + 1) * W + i] = err;
                        if (((i + 1) & 31) == 0 || i == W - 1) {
                            __threadfence_block();
                            ((volatile int*)prog)[rb + 1] = i + 1;
                        }
                    }
                }
                ri = ri == 95 ? 0 : ri + 1;
            }
        }
        if (failed) return;
        __syncwarp();
        for (int c = max(0, nwin - 3); c < nch; ++c) copy_out(c);   // chunks not copied in the loop
        if (row_ok) rowcnt[j] = cnt;
    }
}

// Exclusive prefix of the per-row counts (one CTA); total -> *count.
__global__ void __launch_bounds__(1024) row_scan_kernel(const int* __restrict__ rowcnt, int H,
                                                        int* __restrict__ rowoff, int* count, const int* status) {
    if (*(volatile const int*)status & LOC_DEV_ERR_TIMEOUT) {   // the dithering gave up: no samples
        if (threadIdx.x == 0) *count = 0;
        return;
    }
    __shared__ int part[1024];
    const int per = (H + 1023) / 1024;
    const int j0 = threadIdx.x * per;
    int s = 0;
    for (int j = j0; j < j0 + per && j < H; ++j) s += rowcnt[j];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {            // inclusive Hillis-Steele scan
        const int v = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    int run = threadIdx.x > 0 ? part[threadIdx.x - 1] : 0;
    for (int j = j0; j < j0 + per && j < H; ++j) {
        rowoff[j] = run;
        run += rowcnt[j];
    }
    if (threadIdx.x == 1023) *count = part[1023];
}

// Linear indices of the selected cells in raster order (one warp per row), at most cap.
__global__ void __launch_bounds__(NT) compact_kernel(const uint8_t* __restrict__ sel, const int* __restrict__ rowoff,
                                                     int H, int W, int cap, int32_t* __restrict__ out,
                                                     const int* status) {
    if (*(volatile const int*)status & LOC_DEV_ERR_TIMEOUT) return;   // no row offsets were made
    const int lane = threadIdx.x & 31;
    for (int j = (blockIdx.x * NT + threadIdx.x) >> 5; j < H; j += (gridDim.x * NT) >> 5) {
        int base = rowoff[j];
        for (int i0 = 0; i0 < W; i0 += 32) {
            const int i = i0 + lane;
            const bool on = i < W && sel[(size_t)j * W + i];
            const unsigned int ball = __ballot_sync(0xffffffffu, on);
            const int pos = base + __popc(ball & ((1u << lane) - 1u));
            if (on && pos >= 0 && pos < cap) out[pos] = j * W + i;
            base += __popc(ball);
        }
    }
}

// ------------------------------------------------------------------ ray casting + scoring

// Ranges for given cells and directions (the loc_ray_ranges entry point).
__global__ void __launch_bounds__(NT) ray_ranges_kernel(const uint8_t* __restrict__ trav, int H, int W,
                                                        const int32_t* __restrict__ cells, int n_cells,
                                                        const float* __restrict__ dirs, int n_dirs, float rmax,
                                                        float cell_m, float* __restrict__ out) {
    const size_t n = (size_t)n_cells * n_dirs;
    for (size_t q = (size_t)blockIdx.x * NT + threadIdx.x; q < n; q += (size_t)gridDim.x * NT) {
        const int c = (int)(q / n_dirs), d = (int)(q % n_dirs);
        const int cell = cells[c];
        const float t = dda_cells(trav, H, W, cell / W, cell % W, dirs[2 * d], dirs[2 * d + 1], rmax);
        out[q] = __fmul_rn(t, cell_m);
    }
}

// Order-preserving map of floats to unsigned ints (for atomicMax on floats).
__device__ __forceinline__ unsigned int f2ord(float f) {
    const unsigned int u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ord2f(unsigned int u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7FFFFFFFu) : ~u);
}

// The map as bits: bit b of word w of row j is 1 when cell (j, 32 w + b) is free (words per row
// wb = ceil(W / 32); bits past W are 0).
__global__ void __launch_bounds__(NT) pack_bits_kernel(const uint8_t* __restrict__ trav, int H, int W, int wb,
                                                       uint32_t* __restrict__ bits) {
    const size_t n = (size_t)H * wb;
    for (size_t q = (size_t)blockIdx.x * NT + threadIdx.x; q < n; q += (size_t)gridDim.x * NT) {
        const int j = (int)(q / wb), w = (int)(q % wb);
        uint32_t v = 0;
        for (int b = 0; b < 32; ++b) {
            const int i = 32 * w + b;
            if (i < W && trav[(size_t)j * W + i]) v |= 1u << b;
        }
        bits[q] = v;
    }
}

// One CTA per sampled cell (grid-stride): cast the n_dirs distinct rays once, then for every
// bin k: logL[s][k] = -sum_b (z_b - r(dir_of[k][b]))^2 / (2 sigma^2) over the used beams.
// With WIN the CTA first copies the map bits within R = ceil(rmax) + 2 cells of the sampled
// cell into shared memory (every cell a walk capped at rmax can look at), so each step of the
// walk reads shared memory instead of global memory; the walk itself is the same.
template <bool WIN>
__global__ void __launch_bounds__(kScoreNT) score_kernel(const uint8_t* __restrict__ trav, const uint32_t* __restrict__ bits,
                                                   int wb, int R, int wwin, int H, int W, int K,
                                                   const int32_t* __restrict__ samples, const int* count_ptr, int cap,
                                                   const float* __restrict__ dirs, int n_dirs,
                                                   const int32_t* __restrict__ dir_of, const float* __restrict__ z,
                                                   int n_used, float rmax, float cell_m, float inv2s2,
                                                   float* __restrict__ logL) {
    extern __shared__ float rh[];                 // n_dirs expected ranges (metres), then the window
    uint32_t* win = reinterpret_cast<uint32_t*>(rh + ((n_dirs + 3) & ~3));
    const int n = min(*count_ptr, cap);
    for (int s = blockIdx.x; s < n; s += gridDim.x) {
        const int cell = samples[s];
        const int j = cell / W, i = cell % W;
        if constexpr (WIN) {
            const int j0 = max(0, j - R), j1 = min(H - 1, j + R);
            const int w0 = max(0, i - R) >> 5, w1 = min(W - 1, i + R) >> 5;
            const int rows = j1 - j0 + 1, words = w1 - w0 + 1;
            for (int q = threadIdx.x; q < rows * words; q += kScoreNT) {
                const int r = q / words, c = q % words;
                win[r * wwin + c] = bits[(size_t)(j0 + r) * wb + w0 + c];
            }
            __syncthreads();
            const auto free_at = [win, j0, w0, wwin](int jj, int ii) {
                return ((win[(jj - j0) * wwin + ((ii >> 5) - w0)] >> (ii & 31)) & 1u) != 0u;
            };
            for (int d = threadIdx.x; d < n_dirs; d += kScoreNT)
                rh[d] = __fmul_rn(dda_walk(free_at, H, W, j, i, dirs[2 * d], dirs[2 * d + 1], rmax), cell_m);
        } else {
            for (int d = threadIdx.x; d < n_dirs; d += kScoreNT)
                rh[d] = __fmul_rn(dda_cells(trav, H, W, j, i, dirs[2 * d], dirs[2 * d + 1], rmax), cell_m);
        }
        __syncthreads();
        // one warp per bin: lane l sums the beams b = l, l + 32, ... in order, then a fixed
        // shuffle tree adds the lanes
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        for (int k = warp; k < K; k += kScoreNT / 32) {
            const int32_t* row = dir_of + (size_t)k * n_used;
            float acc = 0.0f;
            for (int b = lane; b < n_used; b += 32) {
                const float e = z[b] - rh[row[b]];
                acc = fmaf(e, e, acc);
            }
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
            if (lane == 0) logL[(size_t)s * K + k] = -acc * inv2s2;
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ Eq. 9 on the sampled set

struct ReweightScalars {
    double mass, wmass, factor;                   // sum b, sum b w over the set; mass / wmass
    unsigned int counter;
    int pad;
};

// Eq. 9 on the sampled set keeps its mass A = sum b and gives b' = A b L / sum(b L).  It is
// evaluated in the log domain against the offset c = max over the set of (log L + log b), so
// every weight w = exp(log L + log b - c) lies in (0, 1] with the largest equal to 1 and the
// normaliser sum w is at least 1: a scan whose likelihood peaks on states of tiny or zero
// belief cannot underflow the normaliser or overflow the factor.  States with b = 0 stay 0.
// reweight_max writes c (as an ordered uint; untouched when no state of the set holds mass).
template <typename T>
__global__ void __launch_bounds__(NT) reweight_max_kernel(const T* __restrict__ B, size_t hw, int K,
                                                          const int32_t* __restrict__ samples, const int* count_ptr,
                                                          int cap, const float* __restrict__ logL, unsigned int* maxL) {
    const int n = min(*count_ptr, cap);
    float best = -FLT_MAX;
    const size_t total = (size_t)n * K;
    for (size_t q = (size_t)blockIdx.x * NT + threadIdx.x; q < total; q += (size_t)gridDim.x * NT) {
        const int s = (int)(q / K), k = (int)(q % K);
        const float b = Store<T>::ld(B + (size_t)k * hw + samples[s]);
        if (b > 0.0f) best = fmaxf(best, logL[q] + logf(b));
    }
    for (int o = 16; o > 0; o >>= 1) best = fmaxf(best, __shfl_down_sync(0xffffffffu, best, o));
    if ((threadIdx.x & 31) == 0 && best > -FLT_MAX) atomicMax(maxL, f2ord(best));
}

// Sums over the sampled states (stored units): mass = sum b, wmass = sum w (the weights above);
// the last CTA writes factor = mass / wmass (0: leave the set as it is).
template <typename T>
__global__ void __launch_bounds__(NT) reweight_sums_kernel(const T* __restrict__ B, size_t hw, int K,
                                                           const int32_t* __restrict__ samples, const int* count_ptr,
                                                           int cap, const float* __restrict__ logL,
                                                           const unsigned int* maxL, double* partials,
                                                           ReweightScalars* rs) {
    __shared__ double red[NT / 32];
    __shared__ double red2[NT / 32];
    const int n = min(*count_ptr, cap);
    const double mx = (double)ord2f(*maxL);
    const bool any = isfinite(mx);                // some state of the set holds mass
    double m = 0.0, wm = 0.0;
    const size_t total = (size_t)n * K;
    for (size_t q = (size_t)blockIdx.x * NT + threadIdx.x; q < total && any; q += (size_t)gridDim.x * NT) {
        const int s = (int)(q / K), k = (int)(q % K);
        const double b = (double)Store<T>::ld(B + (size_t)k * hw + samples[s]);
        m += b;
        if (b > 0.0) wm += exp((double)logL[q] + log(b) - mx);
    }
    const double bm = block_sum<NT>(m, red);
    const double bw = block_sum<NT>(wm, red2);
    __shared__ int s_last;
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = bm;
        partials[2 * blockIdx.x + 1] = bw;
        __threadfence();
        s_last = atomicAdd(&rs->counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double a = 0.0, c = 0.0;
    for (unsigned int b = threadIdx.x; b < gridDim.x; b += NT) {
        a += ((volatile double*)partials)[2 * b];
        c += ((volatile double*)partials)[2 * b + 1];
    }
    const double A = block_sum<NT>(a, red), C = block_sum<NT>(c, red2);
    if (threadIdx.x == 0) {
        rs->counter = 0u;
        rs->mass = A;
        rs->wmass = C;
        rs->factor = (C > 0.0 && isfinite(C) && A > 0.0) ? A / C : 0.0;
    }
}

// The new values b w factor of the sampled states, all (sample, bin) pairs in parallel: FP64
// exp and log, rounded to FP32 and written over logL (which they replace for the store below).
template <typename T>
__global__ void __launch_bounds__(NT) reweight_values_kernel(const T* __restrict__ B, size_t hw, int K,
                                                             const int32_t* __restrict__ samples,
                                                             const int* count_ptr, int cap, float* __restrict__ logL,
                                                             const unsigned int* maxL, const ReweightScalars* rs) {
    const double factor = rs->factor;
    if (!(factor > 0.0)) return;
    const int n = min(*count_ptr, cap);
    const double mx = (double)ord2f(*maxL);
    const size_t total = (size_t)n * K;
    for (size_t q = (size_t)blockIdx.x * NT + threadIdx.x; q < total; q += (size_t)gridDim.x * NT) {
        const int s = (int)(q / K), k = (int)(q % K);
        const size_t at = (size_t)k * hw + samples[s];
        // the new values sum to the set's old mass, so each is finite and at most that mass
        const double b = (double)Store<T>::ld(B + at);
        logL[q] = b > 0.0 ? (float)(factor * exp((double)logL[q] + log(b) - mx)) : 0.0f;
    }
}

// Stores the new values (one thread per sampled cell, its bins in order: the BF16 rounding
// residual runs along theta); the last CTA updates Z by the change of the set's sum.
template <typename T>
__global__ void __launch_bounds__(NT) reweight_apply_kernel(T* __restrict__ B, size_t hw, int K,
                                                            const int32_t* __restrict__ samples, const int* count_ptr,
                                                            int cap, const float* __restrict__ vals,
                                                            ReweightScalars* rs, double* partials, SessionDev* sd) {
    __shared__ double red[NT / 32];
    const double factor = rs->factor;
    const int n = min(*count_ptr, cap);
    KahanF acc;
    if (factor > 0.0) {
        for (int s = blockIdx.x * NT + threadIdx.x; s < n; s += gridDim.x * NT) {
            const size_t cell = (size_t)samples[s];
            const float* v = vals + (size_t)s * K;
            float res = 0.0f;
#pragma unroll 4
            for (int k = 0; k < K; ++k) acc.add(store_diffused<T>(B + (size_t)k * hw + cell, v[k], res));
        }
    }
    const double bt = block_sum<NT>(acc.value(), red);
    finish_sum<NT>(bt, partials, &sd->counter, gridDim.x, red, [sd, rs, factor](double S) {
        if (factor > 0.0) {
            const double Z = sd->Z - rs->mass + S;
            if (Z > 0.0 && isfinite(Z)) {
                sd->Z = Z;
                sd->inv_Z = (float)(1.0 / Z);
            }
        }
    });
}

unsigned int grid_for(size_t n, unsigned int cap) {
    size_t b = (n + NT - 1) / NT;
    if (b < 1) b = 1;
    return (unsigned int)(b < cap ? b : cap);
}

}  // namespace

size_t reweight_scalars_bytes() { return sizeof(ReweightScalars); }

#define LOC_DISPATCH(storage, CALL)                                                   \
    switch (storage) {                                                                \
        case LOC_F32: { using T = float; CALL; } break;                               \
        case LOC_BF16: { using T = __nv_bfloat16; CALL; } break;                      \
        case LOC_F16: { using T = __half; CALL; } break;                              \
        default: return cudaErrorInvalidValue;                                        \
    }

cudaError_t launch_belief_map(const void* B, int storage, const uint8_t* trav, SessionDev* sd, float inv_uniform,
                              int H, int W, int K, float* m, double* partials, unsigned int nparts,
                              unsigned int* counter, int n_samples, float* fs_out, cudaStream_t st) {
    const size_t hw = (size_t)H * W;
    const unsigned int nb = grid_for(hw, nparts < 2048 ? nparts : 2048);
    const size_t vec = storage == LOC_F32 ? 4 : 8;
    if (hw % vec == 0) {
        const unsigned int nbv = grid_for(hw / vec, nparts < 2048 ? nparts : 2048);
        LOC_DISPATCH(storage, (belief_map_vec_kernel<T, 16 / sizeof(T)><<<nbv, NT, 0, st>>>(
                                  (const T*)B, trav, sd, inv_uniform, hw, K, m, partials, counter, n_samples, fs_out)));
    } else {
        LOC_DISPATCH(storage, (belief_map_kernel<T><<<nb, NT, 0, st>>>((const T*)B, trav, sd, inv_uniform, hw, K, m,
                                                                          partials, counter, n_samples, fs_out)));
    }
    return cudaGetLastError();
}

cudaError_t launch_dither(const float* m, const float* fs, int H, int W, uint8_t* sel, int* rowcnt, int* rowoff,
                          int* count, float* bnd, int* prog, int* status, int cap, int32_t* samples,
                          cudaStream_t st) {
    const int nrb = (H + 31) / 32;
    cudaError_t e = cudaMemsetAsync(prog, 0, sizeof(int) * (size_t)(nrb + 1), st);
    if (e != cudaSuccess) return e;
    const size_t smem = sizeof(float) * kFsWarps * 32 * kFsPitch;
    static bool attr_set[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || !attr_set[dev]) {
        e = cudaFuncSetAttribute(fs_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) attr_set[dev] = true;
    }
    fs_kernel<<<1, kFsWarps * 32, smem, st>>>(m, fs, H, W, sel, rowcnt, bnd, prog, status);
    row_scan_kernel<<<1, 1024, 0, st>>>(rowcnt, H, rowoff, count, status);
    if (samples)
        compact_kernel<<<grid_for((size_t)H * 32, 1024), NT, 0, st>>>(sel, rowoff, H, W, cap, samples, status);
    return cudaGetLastError();
}

cudaError_t set_fs_wait(double seconds, int stall) {
    const unsigned long long ns = (unsigned long long)(seconds * 1e9);
    cudaError_t e = cudaMemcpyToSymbol(g_fs_wait_ns, &ns, sizeof(ns));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_fs_stall, &stall, sizeof(stall));
    return e;
}

cudaError_t launch_ray_ranges(const uint8_t* trav, int H, int W, const int32_t* cells, int n_cells, const float* dirs,
                              int n_dirs, float rmax_cells, float cell_m, float* out, cudaStream_t st) {
    ray_ranges_kernel<<<grid_for((size_t)n_cells * n_dirs, 4096), NT, 0, st>>>(trav, H, W, cells, n_cells, dirs,
                                                                              n_dirs, rmax_cells, cell_m, out);
    return cudaGetLastError();
}

cudaError_t launch_pack_bits(const uint8_t* trav, int H, int W, uint32_t* bits, cudaStream_t st) {
    const int wb = (W + 31) / 32;
    pack_bits_kernel<<<grid_for((size_t)H * wb, 4096), NT, 0, st>>>(trav, H, W, wb, bits);
    return cudaGetLastError();
}

cudaError_t launch_score_reweight(void* B, int storage, const uint8_t* trav, const uint32_t* bits, int H, int W, int K,
                                  const int32_t* samples, const int* count, int cap, const float* dirs, int n_dirs,
                                  const int32_t* dir_of, const float* z, int n_used, float rmax_cells, float cell_m,
                                  float inv2s2, float* logL, unsigned int* maxL, void* rs, double* partials,
                                  unsigned int nparts, SessionDev* sd, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(maxL, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess) return e;
    // the map window (R cells around the sampled cell) in shared memory when it fits
    const int R = (int)ceilf(rmax_cells) + 2;
    const int wwin = (2 * R + 1 + 31) / 32 + 1;
    const size_t rh_bytes = sizeof(float) * (size_t)((n_dirs + 3) & ~3);
    const size_t win_bytes = sizeof(uint32_t) * (size_t)(2 * R + 1) * wwin;
    const bool use_win = bits != nullptr && R < 4096 && rh_bytes + win_bytes <= kScoreWindowBytes;
    const size_t smem = rh_bytes + (use_win ? win_bytes : 0);
    // a grid-stride over the samples: CTAs past the count exit at once, but each still costs a launch
    const unsigned int ns = (unsigned int)(cap < 2048 ? (cap > 0 ? cap : 1) : 2048);
    const int wb = (W + 31) / 32;
    if (use_win) {
        if (smem > 48 * 1024) {
            e = cudaFuncSetAttribute(score_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        score_kernel<true><<<ns, kScoreNT, smem, st>>>(trav, bits, wb, R, wwin, H, W, K, samples, count, cap, dirs, n_dirs,
                                                 dir_of, z, n_used, rmax_cells, cell_m, inv2s2, logL);
    } else {
        if (smem > 48 * 1024) {
            e = cudaFuncSetAttribute(score_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        score_kernel<false><<<ns, kScoreNT, smem, st>>>(trav, bits, wb, R, wwin, H, W, K, samples, count, cap, dirs, n_dirs,
                                                  dir_of, z, n_used, rmax_cells, cell_m, inv2s2, logL);
    }
    const size_t hw = (size_t)H * W;
    const unsigned int half = nparts / 2 < 1024 ? nparts / 2 : 1024;
    const unsigned int nb = grid_for((size_t)cap * K, half > 0 ? half : 1);
    ReweightScalars* r = static_cast<ReweightScalars*>(rs);
    LOC_DISPATCH(storage, (reweight_max_kernel<T><<<nb, NT, 0, st>>>((const T*)B, hw, K, samples, count, cap, logL,
                                                                       maxL)));
    LOC_DISPATCH(storage, (reweight_sums_kernel<T><<<nb, NT, 0, st>>>((const T*)B, hw, K, samples, count, cap, logL,
                                                                        maxL, partials, r)));
    LOC_DISPATCH(storage, (reweight_values_kernel<T><<<nb, NT, 0, st>>>((const T*)B, hw, K, samples, count, cap, logL,
                                                                          maxL, r)));
    const unsigned int nb_cells = grid_for((size_t)cap, half > 0 ? half : 1);
    LOC_DISPATCH(storage, (reweight_apply_kernel<T><<<nb_cells, NT, 0, st>>>((T*)B, hw, K, samples, count, cap, logL,
                                                                               r, partials, sd)));
    return cudaGetLastError();
}

}  // namespace loc
