// Paired-column variant of the tiled propagation passes (Alg. 1 shift, mask, blur, correction).
//
// Every thread works on pairs of cells 32 columns apart: S, X, the mask and the P-pass cells of
// a tile are laid out so that (column c, column c + 32) sit side by side, which makes every
// stencil tap of the x blur an aligned 64-bit pair and lets the x blur, the y blur, the theta
// blur, the y lerp of the shift, the mask and the correction all run on the packed FP32 pipe.
// Per element the arithmetic is the same as in the unpaired passes.  Thread coordinates and
// shared-memory pointers are computed once per tile; a plane costs only its shift.
//
//   S pairs s = 0 .. 35 hold tile columns (s - 2, s + 30);  X pairs p = 0 .. 31 hold (p, p + 32).
//   X(p) = g2 (S(p-2) + S(p+2)) + g1 (S(p-1) + S(p+1)) + g0 S(p), i.e. S pairs p .. p+4.
#pragma once

#include "tiled_common.cuh"

namespace loc {
namespace pairs {

using namespace tiled;

constexpr int SPAIRS = 36;             // S pairs per row

// Raw box width in elements: 76 columns are read at most; the row pitch in 32-bit words (76
// for FP32, 44 for 16-bit types) is 12 mod 32, so S items of different row groups read
// different banks.
template <typename T> __host__ __device__ constexpr int pbw() { return sizeof(T) == 4 ? 76 : 88; }

template <typename T, typename C>
constexpr int praw_stride() {          // elements per raw stage, padded to 128 bytes
    return (int)(((C::RAW_H * pbw<T>() * sizeof(T) + 127) / 128) * 128 / sizeof(T));
}
constexpr int SPW = 76;                // S / mask row pitch in floats (38 pairs; 12 mod 32 banks)
constexpr int XPW = 68;                // X row pitch in floats (34 pairs; 4 mod 32 banks)

// TH tile rows, MR rows per P-pass thread, SR S rows per S item, XP X pairs per X item.
template <int TH_, int MR_, int SR_, int XP_, int NSTAGE_, int MINB_>
struct PCfg {
    static constexpr int TH = TH_, MR = MR_, SR = SR_, XP = XP_, NSTAGE = NSTAGE_, MINB = MINB_;
    static constexpr bool PAIRS = true, PIPE = false;
    static constexpr int NT = (TH / MR) * 32;
    static constexpr int XR = TH + 2 * R;
    static constexpr int RAW_H = XR + 1;
    static constexpr int S_ITEMS = (SPAIRS / 4) * (XR / SR);
    static constexpr int X_ITEMS = (32 / XP) * XR;
    static_assert(XR % SR == 0, "S items tile the halo rows");
    static_assert(S_ITEMS <= NT && X_ITEMS <= NT, "one S item and one X item per thread");
    static_assert(XP % 2 == 0 && 32 % XP == 0, "X items of whole 16-byte groups");
};

template <typename T, typename C>
struct PSmem {
    T raw[C::NSTAGE][praw_stride<T, C>()];  // each stage [RAW_H][pbw], 128-byte aligned
    float S[C::XR][SPW];
    float X[C::XR][XPW];
    float wrap[NWRAP][C::TH][TW];            // pairs [r][2p], [2p+1]
    float mk[C::XR][SPW];
    unsigned long long bar[C::NSTAGE];
    double red[C::NT / 32];
};

// Two cells of a pair, 32 columns apart: FP32 as is, BF16 by error diffusion along theta (res:
// the two cells' residuals, see bf16x2_diffuse), FP16 round-to-nearest; the stored values are
// added to sum.  Cells outside the grid have v = 0 and are not stored.
template <typename T> __device__ __forceinline__ void store_pair(T* p, f2 v, f2& res, bool ok0, bool ok1, f2& sum);
template <> __device__ __forceinline__ void store_pair<float>(float* p, f2 v, f2&, bool ok0, bool ok1, f2& sum) {
    float a, b;
    upk(v, a, b);
    if (ok0) p[0] = a;
    if (ok1) p[32] = b;
    sum = fadd2(sum, v);
}
template <>
__device__ __forceinline__ void store_pair<__nv_bfloat16>(__nv_bfloat16* p, f2 v, f2& res, bool ok0, bool ok1,
                                                          f2& sum) {
    float a, b;
    upk(v, a, b);
    f2 st;
    const uint32_t d = bf16x2_diffuse(a, b, res, st);
    if (ok0) *reinterpret_cast<unsigned short*>(p) = (unsigned short)(d & 0xFFFFu);
    if (ok1) *reinterpret_cast<unsigned short*>(p + 32) = (unsigned short)(d >> 16);
    sum = fadd2(sum, st);
}
template <>
__device__ __forceinline__ void store_pair<__half>(__half* p, f2 v, f2&, bool ok0, bool ok1, f2& sum) {
    float a, b;
    upk(v, a, b);
    const __half ha = __float2half_rn(a), hb = __float2half_rn(b);
    if (ok0) p[0] = ha;
    if (ok1) p[32] = hb;
    sum = fadd2(sum, pk(__half2float(ha), __half2float(hb)));
}

// Per-thread coordinates of the three passes, fixed for a tile.
template <typename T, typename C>
struct PThread {
    bool s_on, x_on;
    int s_raw;                         // raw row offset of the S item's first row (elements)
    int s_pair;                        // first S pair of the S item
    int s_row;                         // first S row of the S item
    int x_row, x_pair;                 // X item: row, first X pair
    int r0, cp;                        // P-pass: first row, pair column
};

// tid: the thread's index among the S/X-pass threads; ptid: among the P-pass threads.
template <typename T, typename C>
__device__ __forceinline__ PThread<T, C> pthread_coords(int tid, int ptid) {
    PThread<T, C> t;
    t.s_on = tid < C::S_ITEMS;
    const int su = tid % (SPAIRS / 4), sg = tid / (SPAIRS / 4);
    t.s_pair = 4 * su;
    t.s_row = C::SR * sg;
    t.s_raw = t.s_row * pbw<T>() + 4 * su;
    t.x_on = tid < C::X_ITEMS;
    t.x_row = tid % C::XR;             // consecutive threads take consecutive rows
    t.x_pair = C::XP * (tid / C::XR);
    t.cp = ptid % 32;
    t.r0 = C::MR * (ptid / 32);
    return t;
}

// S-pass of one item: SR rows of 4 S pairs.  XO = xo mod 4 of the plane; xbase = xo - XO.
template <typename T, typename C, int XO>
__device__ __forceinline__ void s_pass(const T* raw, const float (*mk)[SPW], float (*S)[SPW], const PThread<T, C>& th,
                                       int xbase, float fx, float fy) {
    if (!th.s_on) return;
    const f2 fy2 = pk(fy, fy), gy2 = pk(1.0f - fy, 1.0f - fy);
    const T* rp = raw + th.s_raw + xbase;
    f2 prev[4];
#pragma unroll
    for (int r = 0; r <= C::SR; ++r) {
        float va[8], vb[8];
        load8<T>(rp + r * pbw<T>(), va);        // tile columns 4u-2 ..   (first of each pair)
        load8<T>(rp + r * pbw<T>() + 32, vb);   // tile columns 4u+30 .. (second)
        f2 cur[4];
#pragma unroll
        for (int k = 0; k < 4; ++k)
            cur[k] = pk(fmaf(fx, va[XO + k + 1] - va[XO + k], va[XO + k]),
                        fmaf(fx, vb[XO + k + 1] - vb[XO + k], vb[XO + k]));
        if (r > 0) {
            const int y = th.s_row + r - 1;
            const float4 m0 = *reinterpret_cast<const float4*>(&mk[y][2 * th.s_pair]);
            const float4 m1 = *reinterpret_cast<const float4*>(&mk[y][2 * th.s_pair + 4]);
            const f2 mm[4] = {pk(m0.x, m0.y), pk(m0.z, m0.w), pk(m1.x, m1.y), pk(m1.z, m1.w)};
            f2 o[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) o[k] = fmul2(mm[k], ffma2(fy2, cur[k], fmul2(gy2, prev[k])));
            f2* dst = reinterpret_cast<f2*>(&S[y][2 * th.s_pair]);
            reinterpret_cast<ulonglong2*>(dst)[0] = make_ulonglong2(o[0], o[1]);
            reinterpret_cast<ulonglong2*>(dst)[1] = make_ulonglong2(o[2], o[3]);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) prev[k] = cur[k];
    }
}

// X-pass of one item: XP X pairs of one row.
template <typename T, typename C>
__device__ __forceinline__ void x_pass(const float (*S)[SPW], float (*X)[XPW], const PThread<T, C>& th,
                                       const Taps2& tp) {
    if (!th.x_on) return;
    constexpr int NS = C::XP + 4;
    f2 s[NS];
    const ulonglong2* src = reinterpret_cast<const ulonglong2*>(&S[th.x_row][2 * th.x_pair]);
#pragma unroll
    for (int k = 0; k < NS / 2; ++k) {
        const ulonglong2 v = src[k];
        s[2 * k] = v.x;
        s[2 * k + 1] = v.y;
    }
    ulonglong2* dst = reinterpret_cast<ulonglong2*>(&X[th.x_row][2 * th.x_pair]);
#pragma unroll
    for (int k = 0; k < C::XP; k += 2) {
        f2 o[2];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int q = k + j;
            o[j] = ffma2(tp.g2, fadd2(s[q], s[q + 4]), ffma2(tp.g1, fadd2(s[q + 1], s[q + 3]), fmul2(tp.g0, s[q + 2])));
        }
        dst[k / 2] = make_ulonglong2(o[0], o[1]);
    }
}

// P-pass for plane p with the newest ring slot PH = p mod 7: y blur of the thread's MR rows of
// its pair column into the theta ring, then (from p = 6 on) output plane p - 3.
template <typename T, typename C, int PH>
__device__ __forceinline__ void p_pass(const float (*X)[XPW], float (*wrap)[C::TH][TW], const PThread<T, C>& th,
                                       const TileOut& a, const Taps2& tp,
                                       f2 (&ring)[RING][C::MR], const f2 (&cs)[C::MR], f2 (&res)[C::MR], int p,
                                       T* out_tile, size_t plane, int rows, bool ok0, bool ok1, KahanF& acc) {
    constexpr int MR = C::MR;
    const int K = a.K;
    if (p < K) {
        f2 x[MR + 4];
#pragma unroll
        for (int q = 0; q < MR + 4; ++q) x[q] = *reinterpret_cast<const f2*>(&X[th.r0 + q][2 * th.cp]);
#pragma unroll
        for (int rr = 0; rr < MR; ++rr)
            ring[PH][rr] = ffma2(tp.g2, fadd2(x[rr], x[rr + 4]),
                                 ffma2(tp.g1, fadd2(x[rr + 1], x[rr + 3]), fmul2(tp.g0, x[rr + 2])));
        if (p < NWRAP) {
#pragma unroll
            for (int rr = 0; rr < MR; ++rr) *reinterpret_cast<f2*>(&wrap[p][th.r0 + rr][2 * th.cp]) = ring[PH][rr];
        }
    } else {
#pragma unroll
        for (int rr = 0; rr < MR; ++rr) ring[PH][rr] = *reinterpret_cast<const f2*>(&wrap[p - K][th.r0 + rr][2 * th.cp]);
    }
    if (p >= 2 * RT) {
        int o = p - RT;
        if (o >= K) o -= K;
        T* out = out_tile + (size_t)o * plane;
        f2 part = 0ull;
#pragma unroll
        for (int rr = 0; rr < MR; ++rr) {
            f2 t = fmul2(tp.gt[0], ring[(PH + 1) % RING][rr]);
#pragma unroll
            for (int d = 1; d < RING; ++d) t = ffma2(tp.gt[d], ring[(PH + 1 + d) % RING][rr], t);
            const f2 v = fmul2(cs[rr], t);
            const bool in = rr < rows;
            store_pair<T>(out + (size_t)rr * a.W, v, res[rr], in && ok0, in && ok1, part);
        }
        float p0, p1;
        upk(part, p0, p1);
        acc.add(p0 + p1);
    }
}

// One TH x 64 tile, all channels (every thread of the CTA takes part); see tiled::run_tile for
// gp0, p_stop and next_issue.
template <typename T, typename C>
__device__ __forceinline__ bool run_tile(PSmem<T, C>& sm, const TileJob& j, unsigned int gp0, KahanF& acc,
                                         int& p_stop, int& next_issue) {
    constexpr int NT = C::NT, MR = C::MR, NSTAGE = C::NSTAGE, XR = C::XR;
    constexpr int PBW = pbw<T>();
    constexpr uint32_t kBoxBytes = C::RAW_H * PBW * sizeof(T);
    const int tid = threadIdx.x;
    const int H = j.o.H, W = j.o.W, K = j.o.K;
    const int ty0 = j.ty0, tx0 = j.tx0;
    const int reinit = j.reinit;
    const PThread<T, C> th = pthread_coords<T, C>(tid, tid);

    // mask pairs over the halo rows: mk[y][2s] = M(ty0-2+y, tx0+s-2), mk[y][2s+1] = M(.., tx0+s+30)
    for (int q = tid; q < XR * SPAIRS * 2; q += NT) {
        const int y = q / (2 * SPAIRS), e = q % (2 * SPAIRS);
        const int gy = ty0 - R + y, gx = tx0 + (e >> 1) - R + ((e & 1) ? 32 : 0);
        sm.mk[y][e] = (gy >= 0 && gy < H && gx >= 0 && gx < W && j.trav[(size_t)gy * W + gx]) ? 1.0f : 0.0f;
    }
    __syncthreads();
    auto issue = [&](int q) {          // TMA of plane q (thread 0 only)
        const Shift s = j.sh[q];
        int x_al, xo;
        box_x<T>(tx0, s, x_al, xo);
        const unsigned int g = gp0 + (unsigned int)q;
        unsigned long long* b = &sm.bar[g % NSTAGE];
        bar_expect(b, kBoxBytes);
        tma_load(&sm.raw[g % NSTAGE][0], j.tmap, b, x_al, ty0 - R + s.oy, q);
    };
    next_issue = 0;
    if (!reinit) {
        next_issue = NSTAGE < K ? NSTAGE : K;
        if (tid == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            for (int q = 0; q < next_issue; ++q) issue(q);
        }
    }
    // the thread's output cells: rows ty0 + r0 .., columns tx0 + cp and tx0 + cp + 32
    const int gx0 = tx0 + th.cp;
    const bool ok0 = gx0 < W, ok1 = gx0 + 32 < W;
    const int gy0 = ty0 + th.r0;
    const int rows = H - gy0;
    f2 cs[MR];
#pragma unroll
    for (int rr = 0; rr < MR; ++rr) {
        const int gy = gy0 + rr;
        float c0 = 0.0f, c1 = 0.0f;
        if (gy < H) {
            if (ok0) c0 = j.corr[(size_t)gy * W + gx0] * j.in_scale;
            if (ok1) c1 = j.corr[(size_t)gy * W + gx0 + 32] * j.in_scale;
        }
        cs[rr] = pk(c0, c1);
    }
    const size_t plane = (size_t)H * W;
    const size_t cell0 = (size_t)(gy0 < H ? gy0 : 0) * W + gx0;           // plane-0 index of the first cell
    T* out_tile = static_cast<T*>(j.o.B_out) + cell0;
    Taps2 tp;
    tp.g0 = pk(j.g0, j.g0);
    tp.g1 = pk(j.g1, j.g1);
    tp.g2 = pk(j.g2, j.g2);
#pragma unroll
    for (int d = 0; d < RING; ++d) tp.gt[d] = pk(j.gt[d], j.gt[d]);
    f2 ring[RING][MR], res[MR];
#pragma unroll
    for (int d = 0; d < RING; ++d)
#pragma unroll
        for (int k = 0; k < MR; ++k) ring[d][k] = 0ull;
#pragma unroll
    for (int k = 0; k < MR; ++k) res[k] = 0ull;
    int failed = 0;
    int p = 0;
    for (; p < K + NWRAP; ++p) {
        if (p < K) {
            const unsigned int g = gp0 + (unsigned int)p;
            const int stage = g % NSTAGE;
            const Shift s = j.sh[p];
            int x_al, xo;
            box_x<T>(tx0, s, x_al, xo);
            if (reinit) {
                // the uniform input, written where TMA would have put the tile (M as 0/1)
                const int y0 = ty0 - R + s.oy;
                for (int q = tid; q < C::RAW_H * PBW; q += NT) {
                    const int y = q / PBW, c = q % PBW;
                    const int gy = y0 + y, gx = x_al + c;
                    float v = 0.0f;
                    if (gy >= 0 && gy < H && gx >= 0 && gx < W) v = (float)j.trav[(size_t)gy * W + gx];
                    sm.raw[stage][y * PBW + c] = T(v);
                }
                __syncthreads();
            } else if (!bar_wait(&sm.bar[stage], (g / NSTAGE) & 1u)) {
                failed = 1;
            }
            if (!failed) {
                const int xb = xo & ~3;
                switch (xo & 3) {
                    case 0: s_pass<T, C, 0>(sm.raw[stage], sm.mk, sm.S, th, xb, s.fx, s.fy); break;
                    case 1: s_pass<T, C, 1>(sm.raw[stage], sm.mk, sm.S, th, xb, s.fx, s.fy); break;
                    case 2: s_pass<T, C, 2>(sm.raw[stage], sm.mk, sm.S, th, xb, s.fx, s.fy); break;
                    default: s_pass<T, C, 3>(sm.raw[stage], sm.mk, sm.S, th, xb, s.fx, s.fy); break;
                }
            }
            if (__syncthreads_or(failed)) {
                failed = 1;
                break;
            }
            if (!reinit && p + NSTAGE < K) {
                if (tid == 0) {
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    issue(p + NSTAGE);
                }
                next_issue = p + NSTAGE + 1;
            }
            x_pass<T, C>(sm.S, sm.X, th, tp);
            __syncthreads();
        }
        switch (p % RING) {
            case 0: p_pass<T, C, 0>(sm.X, sm.wrap, th, j.o, tp, ring, cs, res, p, out_tile, plane, rows, ok0, ok1, acc); break;
            case 1: p_pass<T, C, 1>(sm.X, sm.wrap, th, j.o, tp, ring, cs, res, p, out_tile, plane, rows, ok0, ok1, acc); break;
            case 2: p_pass<T, C, 2>(sm.X, sm.wrap, th, j.o, tp, ring, cs, res, p, out_tile, plane, rows, ok0, ok1, acc); break;
            case 3: p_pass<T, C, 3>(sm.X, sm.wrap, th, j.o, tp, ring, cs, res, p, out_tile, plane, rows, ok0, ok1, acc); break;
            case 4: p_pass<T, C, 4>(sm.X, sm.wrap, th, j.o, tp, ring, cs, res, p, out_tile, plane, rows, ok0, ok1, acc); break;
            case 5: p_pass<T, C, 5>(sm.X, sm.wrap, th, j.o, tp, ring, cs, res, p, out_tile, plane, rows, ok0, ok1, acc); break;
            default: p_pass<T, C, 6>(sm.X, sm.wrap, th, j.o, tp, ring, cs, res, p, out_tile, plane, rows, ok0, ok1, acc); break;
        }
    }
    p_stop = p;
    // the wrap planes and the X plane are read again by the next tile's first passes
    __syncthreads();
    return !failed;
}

}  // namespace pairs
}  // namespace loc
