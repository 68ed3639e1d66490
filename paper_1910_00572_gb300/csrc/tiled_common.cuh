// Building blocks of the tiled propagation kernels (single session, warp-specialised and
// batched): tile configurations, shared-memory layouts, TMA/mbarrier helpers, packed FP32
// helpers and the S-, X- and P-passes.  Included by step_tiled.cu and batch.cu; step_aniso.cu
// uses its TMA and mbarrier helpers.
#pragma once
#include <cuda.h>

#include <cfloat>
#include <climits>

#include "kernels.h"

namespace loc {
namespace tiled {

constexpr int R = 2, RT = 3;           // kernel radii this kernel is built for
constexpr int TW = 64;                 // tile width (cells)
constexpr int SW = 76;                 // S row pitch (68 used: tile cols -2 .. 65; 76 = 12 mod 32
                                       // banks, so 8 consecutive rows hit 8 distinct bank groups)
constexpr int MW = 76;                 // mask row pitch (floats, same bank spread as S)
constexpr int XW_PITCH = 68;           // X row pitch (64 used; 68 = 4 mod 32 banks)
constexpr int BW = 80;                 // raw box width in elements (76 needed + alignment)
constexpr int RING = 2 * RT + 1;       // 7
constexpr int NWRAP = 2 * RT;          // 6 planes kept for the circular wrap
constexpr unsigned long long kWaitNs = 200ull * 1000 * 1000;   // bounded mbarrier wait

// TH tile rows, MR rows per P-pass thread (2 columns each), SR S-pass rows per item, XW
// X-pass columns per item, NSTAGE raw stages, MINB CTAs per SM asked of the compiler.  PIPE
// runs the passes as a software pipeline over the planes (run_tile_pipe).
template <int TH_, int MR_, int SR_, int XW_, int NSTAGE_, int MINB_, bool PIPE_ = false>
struct Cfg {
    static constexpr int TH = TH_, MR = MR_, SR = SR_, XW = XW_, NSTAGE = NSTAGE_, MINB = MINB_;
    static constexpr bool PAIRS = false, PIPE = PIPE_;
    static constexpr int CR = TH;                  // rows the P-pass threads cover
    static constexpr int NT = (TH / MR) * 32;
    static constexpr int XR = TH + 2 * R;          // rows of S and X
    static constexpr int RAW_H = XR + 1;           // raw rows (bilinear needs one more)
    static_assert(XR % SR == 0, "S-pass row groups must tile the halo rows");
    static_assert((72 / 4) * (XR / SR) <= NT, "one S-pass item per thread");
    static_assert((TW / XW) * XR <= NT, "one X-pass item per thread");
};

struct FastArgs {
    CUtensorMap tmap;                  // X_{t-1} as [K][H][W], box {BW, RAW_H, 1}
    void* B_out;
    const uint8_t* trav;
    const float* corr;
    SessionDev* sd;
    double* partials;
    float* am_pv;                      // per-CTA argmax candidates: value ...
    long long* am_pi;                  // ... and linear index
    long long* am_idx;                 // the argmax of X_t (-1: not produced) ...
    float* am_val;                     // ... and its normalised belief
    float inv_uniform;
    float out_mult;
    double log_out_mult;
    int H, W, K;
    float g0, g1, g2;                  // x/y taps: centre, +-1, +-2
    float gt[RING];                    // theta taps -3 .. +3
    Shift sh[LOC_MAX_K];
};

template <typename T> __host__ __device__ constexpr int align_elems() { return 16 / (int)sizeof(T); }

template <typename T, typename C>
constexpr int raw_stride() {          // elements per raw stage, padded to 128 bytes
    return (int)(((C::RAW_H * BW * sizeof(T) + 127) / 128) * 128 / sizeof(T));
}

template <typename T, typename C>
struct Smem {
    T raw[C::NSTAGE][raw_stride<T, C>()];   // each stage [RAW_H][BW], 128-byte aligned
    float S[C::XR][SW];
    float X[C::XR][XW_PITCH];
    float wrap[NWRAP][C::CR][TW];
    float mk[C::XR][MW];                     // 1 free, 0 occupied / off-grid
    unsigned long long bar[C::NSTAGE];
    double red[C::NT / 32];
};

// The pipelined tile body's shared memory: S and X double-buffered (the S-pass of plane p, the
// X-pass of plane p - 1 and the P-pass of plane p - 2 share one iteration).
template <typename T, typename C>
struct SmemPipe {
    T raw[C::NSTAGE][raw_stride<T, C>()];
    float S[2][C::XR][SW];
    float X[2][C::XR][XW_PITCH];
    float wrap[NWRAP][C::CR][TW];
    float mk[C::XR][MW];
    unsigned long long bar[C::NSTAGE];
    double red[C::NT / 32];
};

__device__ __forceinline__ uint32_t su32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void bar_init(unsigned long long* b, uint32_t n) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(n) : "memory");
}
__device__ __forceinline__ void bar_expect(unsigned long long* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool bar_try(unsigned long long* b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred q;\n mbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n"
        " selp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(ok) : "r"(su32(b)), "r"(parity) : "memory");
    return ok != 0;
}
// Wait for phase `parity` of barrier b; gives up after kWaitNs (returns false).
__device__ __forceinline__ bool bar_wait(unsigned long long* b, uint32_t parity) {
    if (bar_try(b, parity)) return true;
    const unsigned long long t0 = gtimer();
    for (uint32_t it = 0; it < (1u << 26); ++it) {
        if (bar_try(b, parity)) return true;
        if (gtimer() - t0 > kWaitNs) return false;
    }
    return false;
}
__device__ __forceinline__ void tma_load(void* dst, const CUtensorMap* map,
                                         unsigned long long* b, int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(su32(dst)), "l"((unsigned long long)map),
        "r"(su32(b)), "r"(x), "r"(y), "r"(z)
        : "memory");
}

// Packed pairs of FP32 (Blackwell's 2-wide FP32 pipe): lo = first element, hi = second.
typedef unsigned long long f2;
__device__ __forceinline__ f2 pk(float a, float b) {
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void upk(f2 v, float& a, float& b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ f2 fadd2(f2 a, f2 b) {
    f2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 fmul2(f2 a, f2 b) {
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 ffma2(f2 a, f2 b, f2 c) {
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f2 fsub2(f2 a, f2 b) {
    f2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// Compensated (Kahan) FP32 running sums of the two lanes of a packed pair, four packed
// operations per addition; value() widens both to FP64.
struct KahanF2 {
    f2 s = 0ull, c = 0ull;
    __device__ __forceinline__ void add(f2 x) {
        const f2 y = fsub2(x, c);
        const f2 t = fadd2(s, y);
        c = fsub2(fsub2(t, s), y);
        s = t;
    }
    __device__ __forceinline__ double value() const {
        float s0, s1, c0, c1;
        upk(s, s0, s1);
        upk(c, c0, c1);
        return ((double)s0 - (double)c0) + ((double)s1 - (double)c1);
    }
};

// Eight consecutive raw values starting at a 4-element boundary, as FP32.
template <typename T> __device__ __forceinline__ void load8(const T* p, float (&v)[8]);
template <> __device__ __forceinline__ void load8<float>(const float* p, float (&v)[8]) {
    const float4 a = reinterpret_cast<const float4*>(p)[0], b = reinterpret_cast<const float4*>(p)[1];
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}
__device__ __forceinline__ float2 tof2(__nv_bfloat162 h) { return __bfloat1622float2(h); }
__device__ __forceinline__ float2 tof2(__half2 h) { return __half22float2(h); }
template <typename H2, typename T>
__device__ __forceinline__ void load8_16(const T* p, float (&v)[8]) {
    const uint2 a = reinterpret_cast<const uint2*>(p)[0], b = reinterpret_cast<const uint2*>(p)[1];
    const uint32_t w[4] = {a.x, a.y, b.x, b.y};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const H2 h = *reinterpret_cast<const H2*>(&w[k]);
        const float2 f = tof2(h);
        v[2 * k] = f.x;
        v[2 * k + 1] = f.y;
    }
}
template <> __device__ __forceinline__ void load8<__nv_bfloat16>(const __nv_bfloat16* p, float (&v)[8]) {
    load8_16<__nv_bfloat162>(p, v);
}
template <> __device__ __forceinline__ void load8<__half>(const __half* p, float (&v)[8]) {
    load8_16<__half2>(p, v);
}

// Source x of the raw box for a plane: aligned down to 16 bytes; xo = in-box offset of the
// first needed column.
template <typename T>
__device__ __forceinline__ void box_x(int tx0, const Shift& s, int& x_al, int& xo) {
    const int x = tx0 - R + s.ox;
    x_al = x & ~(align_elems<T>() - 1);
    xo = x - x_al;
}

// A thread's S-pass item (4 columns x SR rows of S) and X-pass item (XW columns of one row),
// fixed for the kernel: element offsets into a raw stage, the mask, S and X.
struct SItem {
    int on, raw, mk, s;
};
struct XItem {
    int on, s, x;
};
template <typename C>
__device__ __forceinline__ SItem s_item(int t) {
    constexpr int UNITS = 72 / 4;              // 18 items of 4 columns cover tile cols -2 .. 69
    constexpr int ITEMS = UNITS * (C::XR / C::SR);
    SItem it;
    it.on = t < ITEMS;
    const int u = t % UNITS, y0 = (t / UNITS) * C::SR, c0 = 4 * u;
    it.raw = y0 * BW + c0;
    it.mk = y0 * MW + c0;
    it.s = y0 * SW + c0;
    return it;
}
template <typename C>
__device__ __forceinline__ XItem x_item(int t) {
    constexpr int UNITS = TW / C::XW;
    XItem it;
    it.on = t < UNITS * C::XR;
    const int y = t % C::XR, c0 = C::XW * (t / C::XR);   // consecutive threads take consecutive rows
    it.s = y * SW + c0;
    it.x = y * XW_PITCH + c0;
    return it;
}

// S-pass: S[y][c] for y in [0, XR), c in [0, 72) (tile col c - 2); one item per thread: 4
// columns x SR rows, the x-lerp of the shared raw row carried down.  XO is xo mod 4; the
// runtime part xo - XO (0, or 4 for 16-bit types) moves the base address.  Column pairs run
// on the packed FP32 pipe with the scalar operation order: xl = fx (v1 - v0) + v0, then
// S = m (fy xl + (1 - fy) prev).
template <typename T, typename C, int XO>
__device__ __forceinline__ void s_pass(const T* raw, const float* mk, float* S, const SItem& it, int xbase,
                                       float fx, float fy) {
    if (!it.on) return;
    const f2 fx2 = pk(fx, fx), fy2 = pk(fy, fy);
    const float gy0 = 1.0f - fy;
    const f2 gy2 = pk(gy0, gy0);
    const T* rp = raw + it.raw + xbase;
    const float* mp = mk + it.mk;
    float* sp = S + it.s;
    f2 prev[2];
#pragma unroll
    for (int r = 0; r <= C::SR; ++r) {
        float v[8];
        load8<T>(rp + r * BW, v);
        f2 xl[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const f2 d = pk(v[XO + 2 * k + 1] - v[XO + 2 * k], v[XO + 2 * k + 2] - v[XO + 2 * k + 1]);
            xl[k] = ffma2(fx2, d, pk(v[XO + 2 * k], v[XO + 2 * k + 1]));
        }
        if (r > 0) {
            // one 16-byte mask load (two 8-byte loads 16 bytes apart would conflict 2-way)
            const float4 m = *reinterpret_cast<const float4*>(mp + (r - 1) * MW);
            f2* o2 = reinterpret_cast<f2*>(sp + (r - 1) * SW);
            const f2 o0 = fmul2(pk(m.x, m.y), ffma2(fy2, xl[0], fmul2(gy2, prev[0])));
            const f2 o1 = fmul2(pk(m.z, m.w), ffma2(fy2, xl[1], fmul2(gy2, prev[1])));
            float a, b, c, d;
            upk(o0, a, b);
            upk(o1, c, d);
            *reinterpret_cast<float4*>(o2) = make_float4(a, b, c, d);
        }
        prev[0] = xl[0];
        prev[1] = xl[1];
    }
}

// X-pass: X[y][c0..c0+XW) = x-blur of S, one item (XW columns of one row) per thread, column
// pairs on the packed pipe with the scalar order g2 (s0 + s4) + (g1 (s1 + s3) + g0 s2).
template <typename C>
__device__ __forceinline__ void x_pass(const float* S, float* X, const XItem& it, float g0, float g1, float g2) {
    if (!it.on) return;
    const f2 g02 = pk(g0, g0), g12 = pk(g1, g1), g22 = pk(g2, g2);
    const float* sp = S + it.s;
    float* xp = X + it.x;
    float s[C::XW + 4];
#pragma unroll
    for (int k = 0; k < C::XW + 4; k += 4) {
        const float4 a = *reinterpret_cast<const float4*>(sp + k);
        s[k] = a.x; s[k + 1] = a.y; s[k + 2] = a.z; s[k + 3] = a.w;
    }
#pragma unroll
    for (int k = 0; k < C::XW; k += 4) {
        f2 o[2];
#pragma unroll
        for (int j = 0; j < 4; j += 2) {
            const f2 a = fadd2(pk(s[k + j], s[k + j + 1]), pk(s[k + j + 4], s[k + j + 5]));
            const f2 b = pk(s[k + j + 1] + s[k + j + 3], s[k + j + 2] + s[k + j + 4]);
            const f2 c = pk(s[k + j + 2], s[k + j + 3]);
            o[j / 2] = ffma2(g22, a, ffma2(g12, b, fmul2(g02, c)));
        }
        float a0, a1, b0, b1;
        upk(o[0], a0, a1);
        upk(o[1], b0, b1);
        *reinterpret_cast<float4*>(xp + k) = make_float4(a0, a1, b0, b1);
    }
}

// The S-pass for the in-box offset xo (its residue mod 4 selects the compile-time variant).
template <typename T, typename C>
__device__ __forceinline__ void s_pass_any(const T* raw, const float* mk, float* S, const SItem& it, int xo,
                                           float fx, float fy) {
    const int xb = xo & ~3;
    switch (xo & 3) {
        case 0: s_pass<T, C, 0>(raw, mk, S, it, xb, fx, fy); break;
        case 1: s_pass<T, C, 1>(raw, mk, S, it, xb, fx, fy); break;
        case 2: s_pass<T, C, 2>(raw, mk, S, it, xb, fx, fy); break;
        default: s_pass<T, C, 3>(raw, mk, S, it, xb, fx, fy); break;
    }
}

// Store two neighbouring outputs v = {a, b} (FP32 as is, BF16 by error diffusion along theta,
// FP16 round-to-nearest), add the stored values to sum, and return them as FP32 in st.  res
// holds the BF16 residuals of the two cells (see store2<__nv_bfloat16>); FP32 and FP16 ignore it.
template <typename T> __device__ __forceinline__ void store2(T* p, f2 v, f2& res, f2& sum, f2& st);
template <> __device__ __forceinline__ void store2<float>(float* p, f2 v, f2&, f2& sum, f2& st) {
    *reinterpret_cast<f2*>(p) = v;
    sum = fadd2(sum, v);
    st = v;
}
// BF16 rounding by error diffusion along theta.  Every cell carries a residual from one output
// plane to the next (its own states in plane order): the stored value is the BF16 neighbour of v
// -- the largest BF16 value <= v or the next one above it -- that lies nearest to v + residual,
// and the new residual is (v + residual) - stored.  Each stored value stays within one BF16 unit
// in the last place of its own exact value, and a cell's states keep their total mass to within
// the last residual, so rounding no longer random-walks the mass of concentrated hypotheses from
// step to step (stochastic rounding, unbiased per value, did: its error variance accumulates).
__device__ __forceinline__ uint32_t bf16x2_diffuse(float a, float b, f2& res, f2& st) {
    const f2 w = fadd2(pk(a, b), res);
    float wa, wb;
    upk(w, wa, wb);
    uint32_t rn;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(rn) : "f"(wb), "f"(wa));      // {a, b} in memory order
    const uint32_t lo = __byte_perm(__float_as_uint(a), __float_as_uint(b), 0x7632);   // truncations
    const uint32_t hi = lo + 0x00010001u;                                       // the values above
    // clamp the nearest value of v + residual into [lo, hi]; as signed 16-bit halves a negative
    // v + residual orders below every non-negative value
    const uint32_t d = __vmins2(__vmaxs2(rn, lo), hi);
    st = pk(__uint_as_float(d << 16), __uint_as_float(d & 0xFFFF0000u));
    res = fsub2(w, st);
    return d;
}
template <> __device__ __forceinline__ void store2<__nv_bfloat16>(__nv_bfloat16* p, f2 v, f2& res, f2& sum,
                                                                  f2& st) {
    float a, b;
    upk(v, a, b);
    *reinterpret_cast<uint32_t*>(p) = bf16x2_diffuse(a, b, res, st);
    sum = fadd2(sum, st);
}
template <> __device__ __forceinline__ void store2<__half>(__half* p, f2 v, f2&, f2& sum, f2& st) {
    float a, b;
    upk(v, a, b);
    const __half2 hv = __floats2half2_rn(a, b);
    *reinterpret_cast<__half2*>(p) = hv;
    st = pk(__low2float(hv), __high2float(hv));
    sum = fadd2(sum, st);
}

// Running argmax of the stored values: the larger value, then the lower linear index (the
// order of the argmax pass over the stored tensor).
struct ArgBest {
    float v = -FLT_MAX;
    long long i = LLONG_MAX;
};
__device__ __forceinline__ bool am_better(float v, long long i, float bv, long long bi) {
    return v > bv || (v == bv && i < bi);
}

// The CTA's best (value, index) by a fixed shuffle tree and warp order; valid in thread 0.
// sv / si hold NT/32 entries.
template <int NT>
__device__ __forceinline__ ArgBest am_block(ArgBest b, float* sv, long long* si) {
    for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_down_sync(0xffffffffu, b.v, o);
        const long long oi = __shfl_down_sync(0xffffffffu, b.i, o);
        if (am_better(ov, oi, b.v, b.i)) {
            b.v = ov;
            b.i = oi;
        }
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();                    // an earlier call may still read sv / si
    if (lane == 0) {
        sv[warp] = b.v;
        si[warp] = b.i;
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int w = 1; w < NT / 32; ++w)
            if (am_better(sv[w], si[w], b.v, b.i)) {
                b.v = sv[w];
                b.i = si[w];
            }
    return b;
}

// finish_sum for the normaliser, together with the argmax of the stored tensor: every CTA
// also stores its best (value, index); the CTA that arrives last combines the candidates in a
// fixed order and writes the index and the normalised value (value / Z) to out_idx / out_val,
// the results of the argmax pass over X_t.  When Z is not positive and finite the session
// restarts (its belief reads as uniform over free cells) and out_idx gets -1: no result.
template <int NT, typename Fin>
__device__ __forceinline__ void finish_sum_am(double block_total, ArgBest best, double* partials, float* apv,
                                              long long* api, unsigned int* counter, unsigned int nblocks,
                                              double* red, long long* out_idx, float* out_val, Fin fin) {
    __shared__ int s_last;
    __shared__ float s_v[NT / 32];
    __shared__ long long s_i[NT / 32];
    best = am_block<NT>(best, s_v, s_i);
    if (threadIdx.x == 0) {
        const unsigned int b = blockIdx.x + gridDim.x * blockIdx.y;
        partials[b] = block_total;
        apv[b] = best.v;
        api[b] = best.i;
        __threadfence();
        s_last = atomicAdd(counter, 1u) == nblocks - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double s = 0.0;
    ArgBest g;
    for (unsigned int b = threadIdx.x; b < nblocks; b += NT) {
        s += ((volatile double*)partials)[b];
        const float v = ((volatile float*)apv)[b];
        const long long i = ((volatile long long*)api)[b];
        if (am_better(v, i, g.v, g.i)) {
            g.v = v;
            g.i = i;
        }
    }
    const double tot = block_sum<NT>(s, red);
    g = am_block<NT>(g, s_v, s_i);
    if (threadIdx.x == 0) {
        *counter = 0u;
        fin(tot);
        if (tot > 0.0 && isfinite(tot)) {
            *out_idx = g.i;
            *out_val = (float)((double)g.v / tot);
        } else {
            *out_idx = -1;
        }
    }
}

// Where the P-pass writes: the output tensor and the grid.
struct TileOut {
    void* B_out;
    int H, W, K;
};

// Packed taps of the P-pass.
struct Taps2 {
    f2 g0, g1, g2;                     // y taps {g, g}
    f2 gt[RING];                       // theta taps {g, g}
};

// A P-pass thread's output geometry, fixed for a tile: its first cell's address in plane 0,
// the plane and row strides, the rows inside the grid (and tile).
template <typename T>
struct PCtx {
    T* out0;                           // the thread's first cell (row ty0 + r0, column gx) of plane 0
    size_t plane;                      // H * W elements
    long long base0;                   // linear index of out0 (argmax indices)
    int W;
    int rows;                          // rows of the thread inside the grid and the tile
    bool col_ok;                       // gx < W (both columns: W is even)
    bool full;                         // all MR rows and the columns inside
};

template <typename T, typename C>
__device__ __forceinline__ PCtx<T> p_ctx(const TileOut& a, int r0, int ty0, int gx) {
    PCtx<T> c;
    const long long base = (long long)(ty0 + r0) * a.W + gx;
    c.out0 = static_cast<T*>(a.B_out) + base;
    c.plane = (size_t)a.H * a.W;
    c.base0 = base;
    c.W = a.W;
    int rows = a.H - (ty0 + r0);                       // rows of this thread inside the grid
    if constexpr (C::CR > C::TH) rows = min(rows, C::TH - r0);   // ... and inside the tile
    c.rows = rows;
    c.col_ok = gx < a.W;
    c.full = rows >= C::MR && c.col_ok;
    return c;
}

// P-pass for plane p with the newest ring slot PH = p mod 7.  The thread's cells are rows
// r0 .. r0+MR-1 of the tile, columns 2cp and 2cp+1, handled as column pairs.
// res holds the BF16 rounding residuals of the thread's cells, carried from plane to plane.
// With AM the thread also keeps the running argmax of the values it stores in *am.
template <typename T, typename C, int PH, bool AM = false>
__device__ __forceinline__ void p_pass(const float (*X)[XW_PITCH], float (*wrap)[C::CR][TW],
                                       const PCtx<T>& pc, int K, const Taps2& tp,
                                       f2 (&ring)[RING][C::MR], const f2 (&cs)[C::MR], f2 (&res)[C::MR],
                                       int p, int r0, int cp, KahanF2& acc, ArgBest* am = nullptr) {
    constexpr int MR = C::MR;
    if (p < K) {
        f2 x[MR + 4];
#pragma unroll
        for (int q = 0; q < MR + 4; ++q) x[q] = *reinterpret_cast<const f2*>(&X[r0 + q][2 * cp]);
#pragma unroll
        for (int rr = 0; rr < MR; ++rr)
            ring[PH][rr] = ffma2(tp.g2, fadd2(x[rr], x[rr + 4]),
                                 ffma2(tp.g1, fadd2(x[rr + 1], x[rr + 3]), fmul2(tp.g0, x[rr + 2])));
        if (p < NWRAP) {
#pragma unroll
            for (int rr = 0; rr < MR; ++rr) *reinterpret_cast<f2*>(&wrap[p][r0 + rr][2 * cp]) = ring[PH][rr];
        }
    } else {
#pragma unroll
        for (int rr = 0; rr < MR; ++rr) ring[PH][rr] = *reinterpret_cast<const f2*>(&wrap[p - K][r0 + rr][2 * cp]);
    }
    if (p >= 2 * RT) {
        int o = p - RT;
        if (o >= K) o -= K;
        T* out = pc.out0 + (size_t)o * pc.plane;
        f2 part = 0ull;
        f2 stv[MR];                                    // stored values (-FLT_MAX: not stored)
        if (pc.full) {
#pragma unroll
            for (int rr = 0; rr < MR; ++rr) {
                f2 t = fmul2(tp.gt[0], ring[(PH + 1) % RING][rr]);
#pragma unroll
                for (int d = 1; d < RING; ++d) t = ffma2(tp.gt[d], ring[(PH + 1 + d) % RING][rr], t);
                store2<T>(out + (size_t)rr * pc.W, fmul2(cs[rr], t), res[rr], part, stv[rr]);
            }
        } else {
#pragma unroll
            for (int rr = 0; rr < MR; ++rr) {
                f2 t = fmul2(tp.gt[0], ring[(PH + 1) % RING][rr]);
#pragma unroll
                for (int d = 1; d < RING; ++d) t = ffma2(tp.gt[d], ring[(PH + 1 + d) % RING][rr], t);
                stv[rr] = pk(-FLT_MAX, -FLT_MAX);
                if (rr < pc.rows && pc.col_ok)
                    store2<T>(out + (size_t)rr * pc.W, fmul2(cs[rr], t), res[rr], part, stv[rr]);
            }
        }
        acc.add(part);
        if constexpr (AM) {
            float m = -FLT_MAX;
#pragma unroll
            for (int rr = 0; rr < MR; ++rr) {
                float lo, hi;
                upk(stv[rr], lo, hi);
                m = fmaxf(m, fmaxf(lo, hi));
            }
            if (m >= am->v && m > -FLT_MAX) {          // rare: the lowest index holding m
                const long long base = pc.base0 + (long long)o * (long long)pc.plane;
                long long idx = LLONG_MAX;
#pragma unroll
                for (int rr = 0; rr < MR; ++rr) {
                    float lo, hi;
                    upk(stv[rr], lo, hi);
                    if (idx == LLONG_MAX && lo == m) idx = base + (long long)rr * pc.W;
                    if (idx == LLONG_MAX && hi == m) idx = base + (long long)rr * pc.W + 1;
                }
                if (am_better(m, idx, am->v, am->i)) {
                    am->v = m;
                    am->i = idx;
                }
            }
        }
    }
}

// One tile of the synchronous tiled kernel (every thread of the CTA takes part):
// Algorithm 1's propagation for all channels of a TH x 64 output tile, adding the stored values to acc.
struct TileJob {
    const CUtensorMap* tmap;          // X_{t-1} as [K][H][W]
    const Shift* sh;                  // per-channel source offsets
    TileOut o;
    const uint8_t* trav;
    const float* corr;
    const float* gt;                  // theta taps (7)
    float in_scale;                   // 1/Z (or the uniform value) times the storage multiplier
    float g0, g1, g2;
    int reinit;                       // read the input as M (uniform restart) instead of TMA
    int ty0, tx0;
};

// TMA of plane q of the tile into its raw stage (thread 0 only); gp0 as for run_tile.
template <typename T, typename C, typename SM>
__device__ __forceinline__ void issue_plane(SM& sm, const TileJob& j, unsigned int gp0, int q) {
    constexpr uint32_t kBoxBytes = C::RAW_H * BW * sizeof(T);
    const Shift s = j.sh[q];
    int x_al, xo;
    box_x<T>(j.tx0, s, x_al, xo);
    const unsigned int g = gp0 + (unsigned int)q;
    unsigned long long* b = &sm.bar[g % C::NSTAGE];
    bar_expect(b, kBoxBytes);
    tma_load(&sm.raw[g % C::NSTAGE][0], j.tmap, b, x_al, j.ty0 - R + s.oy, q);
}

// The start of a synchronous tile: the map mask over the halo region (rows ty0-2 .., cols
// tx0-2 ..) into shared memory, and the first planes requested by TMA (none for a restart,
// which reads M).  Returns the number of planes requested.
template <typename T, typename C, typename SM>
__device__ __forceinline__ int tile_start(SM& sm, const TileJob& j, unsigned int gp0) {
    const int H = j.o.H, W = j.o.W, K = j.o.K;
    for (int q = threadIdx.x; q < C::XR * MW; q += C::NT) {
        const int y = q / MW, c = q % MW;
        const int gy = j.ty0 - R + y, gx = j.tx0 - R + c;
        sm.mk[y][c] = (gy >= 0 && gy < H && gx >= 0 && gx < W && j.trav[(size_t)gy * W + gx]) ? 1.0f : 0.0f;
    }
    __syncthreads();                // the S-passes read the whole mask
    if (j.reinit) return 0;
    const int n = C::NSTAGE < K ? C::NSTAGE : K;
    if (threadIdx.x == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        for (int q = 0; q < n; ++q) issue_plane<T, C>(sm, j, gp0, q);
    }
    return n;
}

// A P-pass thread's correction times the input scale, for its rows r0 .. r0+MR-1 and columns
// gxp, gxp+1 (0 outside the grid).
template <typename C>
__device__ __forceinline__ void tile_corr(f2 (&cs)[C::MR], const TileJob& j, int r0, int gxp) {
    const int H = j.o.H, W = j.o.W;
#pragma unroll
    for (int rr = 0; rr < C::MR; ++rr) {
        const int gy = j.ty0 + r0 + rr;
        float c0 = 0.0f, c1 = 0.0f;
        if (gy < H && gxp < W) {
            c0 = j.corr[(size_t)gy * W + gxp] * j.in_scale;
            c1 = j.corr[(size_t)gy * W + gxp + 1] * j.in_scale;
        }
        cs[rr] = pk(c0, c1);
    }
}

__device__ __forceinline__ Taps2 tile_taps(const TileJob& j) {
    Taps2 tp;
    tp.g0 = pk(j.g0, j.g0);
    tp.g1 = pk(j.g1, j.g1);
    tp.g2 = pk(j.g2, j.g2);
#pragma unroll
    for (int d = 0; d < RING; ++d) tp.gt[d] = pk(j.gt[d], j.gt[d]);
    return tp;
}

// gp0: planes this CTA has already loaded through the mbarriers (their phases continue).
// Returns false when a bounded wait gave up; p_stop / next_issue then bound the copies that
// may still be in flight.
template <typename T, typename C>
__device__ __forceinline__ bool run_tile(Smem<T, C>& sm, const TileJob& j, unsigned int gp0, KahanF2& acc,
                                         int& p_stop, int& next_issue) {
    constexpr int NT = C::NT, MR = C::MR, NSTAGE = C::NSTAGE;
    const int tid = threadIdx.x;
    const int H = j.o.H, W = j.o.W, K = j.o.K;
    const int ty0 = j.ty0, tx0 = j.tx0;
    const int reinit = j.reinit;
    next_issue = tile_start<T, C>(sm, j, gp0);
    const int cp = tid % 32, rg = tid / 32;
    const int r0 = MR * rg, gxp = tx0 + 2 * cp;
    f2 cs[MR];
    tile_corr<C>(cs, j, r0, gxp);
    const Taps2 tp = tile_taps(j);
    f2 ring[RING][MR], res[MR];
#pragma unroll
    for (int d = 0; d < RING; ++d)
#pragma unroll
        for (int k = 0; k < MR; ++k) ring[d][k] = 0ull;
#pragma unroll
    for (int k = 0; k < MR; ++k) res[k] = 0ull;
    const PCtx<T> pc = p_ctx<T, C>(j.o, r0, ty0, gxp);
    const SItem si = s_item<C>(tid);
    const XItem xi = x_item<C>(tid);
    int failed = 0;
    int p = 0, ph = 0;                                  // ph = p mod RING
    for (; p < K + NWRAP; ++p, ph = ph == RING - 1 ? 0 : ph + 1) {
        if (p < K) {
            const unsigned int g = gp0 + (unsigned int)p;
            const int stage = g % NSTAGE;
            const Shift s = j.sh[p];
            int x_al, xo;
            box_x<T>(tx0, s, x_al, xo);
            if (reinit) {
                // the uniform input, written where TMA would have put the tile (M as 0/1)
                const int y0 = ty0 - R + s.oy;
                for (int q = tid; q < C::RAW_H * BW; q += NT) {
                    const int y = q / BW, c = q % BW;
                    const int gy = y0 + y, gx = x_al + c;
                    float v = 0.0f;
                    if (gy >= 0 && gy < H && gx >= 0 && gx < W) v = (float)j.trav[(size_t)gy * W + gx];
                    sm.raw[stage][y * BW + c] = T(v);
                }
                __syncthreads();
            } else if (!bar_wait(&sm.bar[stage], (g / NSTAGE) & 1u)) {
                failed = 1;
            }
            if (!failed) {
                s_pass_any<T, C>(sm.raw[stage], &sm.mk[0][0], &sm.S[0][0], si, xo, s.fx, s.fy);
            }
            if (__syncthreads_or(failed)) {
                failed = 1;
                break;
            }
            if (!reinit && p + NSTAGE < K) {
                if (tid == 0) {
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    issue_plane<T, C>(sm, j, gp0, p + NSTAGE);
                }
                next_issue = p + NSTAGE + 1;
            }
            x_pass<C>(&sm.S[0][0], &sm.X[0][0], xi, j.g0, j.g1, j.g2);
            __syncthreads();
        }
        switch (ph) {
            case 0: p_pass<T, C, 0>(sm.X, sm.wrap, pc, K, tp, ring, cs, res, p, r0, cp, acc); break;
            case 1: p_pass<T, C, 1>(sm.X, sm.wrap, pc, K, tp, ring, cs, res, p, r0, cp, acc); break;
            case 2: p_pass<T, C, 2>(sm.X, sm.wrap, pc, K, tp, ring, cs, res, p, r0, cp, acc); break;
            case 3: p_pass<T, C, 3>(sm.X, sm.wrap, pc, K, tp, ring, cs, res, p, r0, cp, acc); break;
            case 4: p_pass<T, C, 4>(sm.X, sm.wrap, pc, K, tp, ring, cs, res, p, r0, cp, acc); break;
            case 5: p_pass<T, C, 5>(sm.X, sm.wrap, pc, K, tp, ring, cs, res, p, r0, cp, acc); break;
            default: p_pass<T, C, 6>(sm.X, sm.wrap, pc, K, tp, ring, cs, res, p, r0, cp, acc); break;
        }
    }
    p_stop = p;
    // the wrap planes and the X plane are read again by the next tile's first passes
    __syncthreads();
    return !failed;
}

// run_tile as a software pipeline over the planes: iteration it runs the S-pass of plane it,
// the X-pass of plane it - 1 and the P-pass of plane it - 2 (each from the buffers the previous
// iteration wrote) and ends with one CTA barrier, where run_tile has two per plane.  The passes
// and their operation order are run_tile's, so the results are bit-identical to the
// synchronous configuration with the same tile.  Same contract as run_tile.
template <typename T, typename C>
__device__ __forceinline__ bool run_tile_pipe(SmemPipe<T, C>& sm, const TileJob& j, unsigned int gp0, KahanF2& acc,
                                              int& p_stop, int& next_issue) {
    constexpr int NT = C::NT, MR = C::MR, NSTAGE = C::NSTAGE;
    const int tid = threadIdx.x;
    const int H = j.o.H, W = j.o.W, K = j.o.K;
    const int ty0 = j.ty0, tx0 = j.tx0;
    const int reinit = j.reinit;
    next_issue = tile_start<T, C>(sm, j, gp0);
    const int cp = tid % 32, rg = tid / 32;
    const int r0 = MR * rg, gxp = tx0 + 2 * cp;
    f2 cs[MR];
    tile_corr<C>(cs, j, r0, gxp);
    const Taps2 tp = tile_taps(j);
    f2 ring[RING][MR], res[MR];
#pragma unroll
    for (int d = 0; d < RING; ++d)
#pragma unroll
        for (int k = 0; k < MR; ++k) ring[d][k] = 0ull;
#pragma unroll
    for (int k = 0; k < MR; ++k) res[k] = 0ull;
    const PCtx<T> pc = p_ctx<T, C>(j.o, r0, ty0, gxp);
    const SItem si = s_item<C>(tid);
    const XItem xi = x_item<C>(tid);
    int failed = 0;
    int ph = 0;                                         // (it - 2) mod RING: the P-pass's ring slot
    int it = 0;
    for (; it < K + NWRAP + 2; ++it) {
        const int ps = it, px = it - 1, pp = it - 2;
        if (ps < K) {
            const unsigned int g = gp0 + (unsigned int)ps;
            const int stage = g % NSTAGE;
            const Shift s = j.sh[ps];
            int x_al, xo;
            box_x<T>(tx0, s, x_al, xo);
            if (reinit) {
                // the uniform input, written where TMA would have put the tile (M as 0/1); every
                // thread takes this branch (the flag is per launch)
                const int y0 = ty0 - R + s.oy;
                for (int q = tid; q < C::RAW_H * BW; q += NT) {
                    const int y = q / BW, c = q % BW;
                    const int gy = y0 + y, gx = x_al + c;
                    float v = 0.0f;
                    if (gy >= 0 && gy < H && gx >= 0 && gx < W) v = (float)j.trav[(size_t)gy * W + gx];
                    sm.raw[stage][y * BW + c] = T(v);
                }
                __syncthreads();
            } else if (!bar_wait(&sm.bar[stage], (g / NSTAGE) & 1u)) {
                failed = 1;
            }
            if (!failed) s_pass_any<T, C>(sm.raw[stage], &sm.mk[0][0], &sm.S[ps & 1][0][0], si, xo, s.fx, s.fy);
        }
        if (px >= 0 && px < K && !failed) x_pass<C>(&sm.S[px & 1][0][0], &sm.X[px & 1][0][0], xi, j.g0, j.g1, j.g2);
        if (pp >= 0 && !failed) {
            const float (*X)[XW_PITCH] = sm.X[pp & 1];
            switch (ph) {
                case 0: p_pass<T, C, 0>(X, sm.wrap, pc, K, tp, ring, cs, res, pp, r0, cp, acc); break;
                case 1: p_pass<T, C, 1>(X, sm.wrap, pc, K, tp, ring, cs, res, pp, r0, cp, acc); break;
                case 2: p_pass<T, C, 2>(X, sm.wrap, pc, K, tp, ring, cs, res, pp, r0, cp, acc); break;
                case 3: p_pass<T, C, 3>(X, sm.wrap, pc, K, tp, ring, cs, res, pp, r0, cp, acc); break;
                case 4: p_pass<T, C, 4>(X, sm.wrap, pc, K, tp, ring, cs, res, pp, r0, cp, acc); break;
                case 5: p_pass<T, C, 5>(X, sm.wrap, pc, K, tp, ring, cs, res, pp, r0, cp, acc); break;
                default: p_pass<T, C, 6>(X, sm.wrap, pc, K, tp, ring, cs, res, pp, r0, cp, acc); break;
            }
            ph = ph == RING - 1 ? 0 : ph + 1;
        }
        // S of plane ps, X of plane px and the P-pass's reads of X are done everywhere
        if (__syncthreads_or(failed)) {
            failed = 1;
            break;
        }
        if (!reinit && ps < K && ps + NSTAGE < K) {   // the stage of plane ps takes plane ps + NSTAGE
            if (tid == 0) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                issue_plane<T, C>(sm, j, gp0, ps + NSTAGE);
            }
            next_issue = ps + NSTAGE + 1;
        }
    }
    p_stop = it < K ? it : K;
    __syncthreads();
    return !failed;
}

}  // namespace tiled
}  // namespace loc
