// Propagation with anisotropic motion noise (Eq. 5-6 with sigma_x != sigma_y): Algorithm 1's
// propagation for all channels plus the Eq. 9 normaliser, any kernel radii up to LOC_MAX_R_XY /
// LOC_MAX_R_THETA and any storage type.
//
// The motion kernel of output channel k is exp(-1/2 [(d . e_k / sigma_x)^2 + (d . n_k /
// sigma_y)^2 + (dk / sigma_theta)^2]) with e_k the channel's heading phi_k = 2 pi k / K +
// theta_t and n_k its normal, normalised to sum 1: separable into the theta taps and a
// rotated, non-separable x/y stencil that differs per channel.  Since every source plane of
// output channel k is blurred with the same x/y stencil, the theta sum is taken first:
//   S_c   = M * bilinear(X_{t-1}[c])                          (Eq. 3 + Algorithm 1's first mask)
//   C_k   = sum_d gt[d] S_{k+d}                               (theta part, circular)
//   T_k   = g_k (x/y) applied to C_k;  G_k = g_k applied to M  (Eq. 7, Eq. 8 for B_0)
//   X_t[k] = M * T_k / G_k * (1 / Z_{t-1})                    (Algorithm 1's mask + edge correction)
// Channel k's stencil is computed in the CTA from phi_k (FP32 sin/cos/exp); its normalisation
// cancels in T_k / G_k.
//
// Layout.  One CTA owns a 32 x 32 tile of output cells and streams the source planes
// kk = -r_th .. K-1+r_th.  Shared memory holds, over the tile plus R rows above and below and
// 4 columns left and right (a 40-column region, so that every 4-cell group is 16-byte
// aligned): the ring of the last 2 r_th + 1 planes S, two buffers of the theta sum C and of
// the channel's stencil, and the map M; and, in the storage type, the raw (shifted) input
// boxes of two planes.
//
// Warp-specialised pipeline.  Six producer warps take plane kk: its input box (one TMA copy
// per plane, x rounded down to 16 bytes, zeros outside the grid, issued two planes ahead,
// where the row pitch allows; else plain loads, and always for the restart input, the map),
// the S pass into the ring and, once the ring is full, C of channel o = kk - r_th and its
// stencil into buffer o mod 3.  A producer always computes S and C for the same region cells,
// so the ring cells it sums are its own writes.  Four consumer warps take channel o from that
// buffer: the stencil, the division by G_k, the store and the Z partial sums.  The hand-offs
// are mbarriers (FULL[b]: the 192 producers arrive after writing; EMPTY[b]: the 128 consumers
// arrive after reading) with bounded waits; the producers also meet at a named barrier
// before a raw box is overwritten.
//
// Each consumer thread owns a 2 x 4 block of output cells (lanes 8 wide x 4 high per warp);
// each stencil row is three 16-byte loads of C (and of M), conflict-free across each 8-lane
// quarter warp, reused by up to 2 x 4 x (2R+1) taps, with the row loop unrolled at compile
// time.  Where every map cell under a warp's stencil windows is free, G_k is the stencil's own
// sum taken in the same order, so the warp skips the M loads and half the FMAs with a
// bit-identical result.
#include <type_traits>

#include "tiled_common.cuh"

namespace loc {
namespace {

using tiled::bar_expect;
using tiled::bar_init;
using tiled::bar_wait;
using tiled::tma_load;

constexpr int TH = 32, TW = 32;
constexpr int NP = 192, NC = 128, NT = NP + NC;  // producer and consumer threads
constexpr int BY = 2;                          // output rows per thread (4 columns each)
constexpr int NBUF = 3;                        // C / stencil buffers between producers and consumers
constexpr int HX = 4;                          // region columns left of the tile
constexpr int RCOLS = TW + 2 * HX;             // 40 region columns
constexpr int P = RCOLS;                       // row pitch of ring, C and M (floats)
constexpr int RAW_COLS = RCOLS + 1;            // 41 input columns per row
constexpr int NG = RCOLS / 4;                  // 4-cell groups per region row

// raw box row pitch in elements of T: 41 columns plus the offset of the first one within its
// 16-byte group (TMA x is rounded down to 16 bytes): 44 FP32, 48 16-bit
template <typename T> __host__ __device__ constexpr int raw_pitch() { return sizeof(T) == 4 ? 44 : 48; }

template <int R>
struct Geo {
    static constexpr int RR = TH + 2 * R;                 // region rows
    static constexpr int RAW_ROWS = RR + 1;
    static constexpr int D = 2 * R + 1;                   // stencil side
    static constexpr int GP = (D + 3) / 4 * 4;            // stencil row pitch
    static constexpr int NR = BY + 2 * R;                 // source rows under a block
};

template <typename T, int R>
__host__ __device__ constexpr size_t raw_buf_bytes() {                        // one raw box, rounded to 128 bytes
    return ((size_t)Geo<R>::RAW_ROWS * raw_pitch<T>() * sizeof(T) + 127) / 128 * 128;
}

template <typename T, int R>
size_t aniso_smem_bytes(int rt) {
    using G = Geo<R>;
    const size_t nring = 2 * (size_t)rt + 1;
    return 2 * raw_buf_bytes<T, R>() + (nring + NBUF + 1) * G::RR * P * sizeof(float) +
           NBUF * (size_t)G::D * G::GP * sizeof(float);
}

template <typename T> __device__ __forceinline__ float to_f(T v);
template <> __device__ __forceinline__ float to_f<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <> __device__ __forceinline__ float to_f<__half>(__half v) { return __half2float(v); }

template <typename T> __device__ __forceinline__ T from_u8(uint8_t v);
template <> __device__ __forceinline__ float from_u8<float>(uint8_t v) { return (float)v; }
template <> __device__ __forceinline__ __nv_bfloat16 from_u8<__nv_bfloat16>(uint8_t v) {
    return __float2bfloat16_rn((float)v);
}
template <> __device__ __forceinline__ __half from_u8<__half>(uint8_t v) { return __float2half_rn((float)v); }

// The stored form of an output value of a cell whose BF16 residual is r (BF16 by error diffusion
// along theta, FP16 round-to-nearest).
template <typename T> __device__ __forceinline__ T round_out(float v, float& r);
template <> __device__ __forceinline__ float round_out<float>(float v, float&) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 round_out<__nv_bfloat16>(float v, float& r) {
    return bf16_diffuse(v, r);
}
template <> __device__ __forceinline__ __half round_out<__half>(float v, float&) { return __float2half_rn(v); }

template <typename T> struct Vec4;
template <> struct Vec4<float> {
    static __device__ __forceinline__ void st(float* p, const float (&v)[4]) {
        *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
};
template <> struct Vec4<__nv_bfloat16> {
    static __device__ __forceinline__ void st(__nv_bfloat16* p, const __nv_bfloat16 (&v)[4]) {
        uint2 u;
        u.x = (uint32_t)__bfloat16_as_ushort(v[0]) | ((uint32_t)__bfloat16_as_ushort(v[1]) << 16);
        u.y = (uint32_t)__bfloat16_as_ushort(v[2]) | ((uint32_t)__bfloat16_as_ushort(v[3]) << 16);
        *reinterpret_cast<uint2*>(p) = u;
    }
};
template <> struct Vec4<__half> {
    static __device__ __forceinline__ void st(__half* p, const __half (&v)[4]) {
        uint2 u;
        u.x = (uint32_t)__half_as_ushort(v[0]) | ((uint32_t)__half_as_ushort(v[1]) << 16);
        u.y = (uint32_t)__half_as_ushort(v[2]) | ((uint32_t)__half_as_ushort(v[3]) << 16);
        *reinterpret_cast<uint2*>(p) = u;
    }
};

__device__ __forceinline__ void ld4(const float* p, float* d) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    d[0] = v.x; d[1] = v.y; d[2] = v.z; d[3] = v.w;
}

// Raw elements p[0 .. NV) as float by aligned vector loads: 8 FP32 (two 16-byte loads, p
// 16-byte aligned) or 12 16-bit (three 8-byte loads, p 8-byte aligned).
template <typename T> struct RawRow;
template <> struct RawRow<float> {
    static constexpr int NV = 8;
    static __device__ __forceinline__ void ld(const float* p, float (&v)[NV]) {
        ld4(p, v);
        ld4(p + 4, v + 4);
    }
};
template <typename H2, float2 (*CVT)(H2)>
__device__ __forceinline__ void ld12_16(const void* p, float (&v)[12]) {
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const uint2 u = reinterpret_cast<const uint2*>(p)[q];
        H2 a, b;
        memcpy(&a, &u.x, 4);
        memcpy(&b, &u.y, 4);
        const float2 fa = CVT(a), fb = CVT(b);
        v[4 * q] = fa.x; v[4 * q + 1] = fa.y; v[4 * q + 2] = fb.x; v[4 * q + 3] = fb.y;
    }
}
__device__ __forceinline__ float2 cvt_bf2(__nv_bfloat162 h) { return __bfloat1622float2(h); }
__device__ __forceinline__ float2 cvt_h2(__half2 h) { return __half22float2(h); }
template <> struct RawRow<__nv_bfloat16> {
    static constexpr int NV = 12;
    static __device__ __forceinline__ void ld(const __nv_bfloat16* p, float (&v)[NV]) {
        ld12_16<__nv_bfloat162, cvt_bf2>(p, v);
    }
};
template <> struct RawRow<__half> {
    static constexpr int NV = 12;
    static __device__ __forceinline__ void ld(const __half* p, float (&v)[NV]) { ld12_16<__half2, cvt_h2>(p, v); }
};

template <int V> using IC = std::integral_constant<int, V>;

__device__ __forceinline__ void bar_arrive(unsigned long long* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tiled::su32(b)) : "memory");
}
// named barrier 1 among the producer threads only (every producer reaches each one)
__device__ __forceinline__ void producers_sync() { asm volatile("bar.sync 1, %0;" ::"n"(NP) : "memory"); }

// The stencil over one 2 x 4 block: t[oy][ox] = sum g[dj][di] C[oy+dj][ox+di] and, unless the
// warp is interior, gm[oy][ox] = sum g[dj][di] M[oy+dj][ox+di], both in row-major tap order.
// `c0` / `m0` point at the block's first source row, 4 - R columns left of its first cell
// rounded down to the 16-byte group (the window is columns 4 - R .. 7 + R of 12).
template <int R, bool WITH_M>
__device__ __forceinline__ void stencil_block(const float* c0, const float* m0, const float* gs,
                                              float (&t)[BY][4], float (&gm)[BY][4]) {
    using G = Geo<R>;
#pragma unroll
    for (int sr = 0; sr < G::NR; ++sr) {
        float c[12], m[12];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            ld4(c0 + sr * P + 4 * q, c + 4 * q);
            if (WITH_M) ld4(m0 + sr * P + 4 * q, m + 4 * q);
        }
#pragma unroll
        for (int oy = 0; oy < BY; ++oy) {
            const int dj = sr - oy;
            if (dj < 0 || dj >= G::D) continue;
            float w[G::GP];
#pragma unroll
            for (int q = 0; q < G::GP / 4; ++q) ld4(gs + dj * G::GP + 4 * q, w + 4 * q);
#pragma unroll
            for (int di = 0; di < G::D; ++di) {
#pragma unroll
                for (int ox = 0; ox < 4; ++ox) {
                    t[oy][ox] = fmaf(w[di], c[ox + di + 4 - R], t[oy][ox]);
                    if (WITH_M) gm[oy][ox] = fmaf(w[di], m[ox + di + 4 - R], gm[oy][ox]);
                }
            }
        }
    }
}

template <typename T, int R>
__global__ void __launch_bounds__(NT, 2) step_aniso_kernel(const __grid_constant__ StepArgs a,
                                                           const __grid_constant__ CUtensorMap tmap,
                                                           int use_tma) {
    using G = Geo<R>;
    constexpr int RPT = raw_pitch<T>();
    constexpr size_t RAW_BUF = raw_buf_bytes<T, R>();
    constexpr int AL = 16 / (int)sizeof(T);              // TMA x alignment in elements
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ double red[NT / 32];
    __shared__ unsigned long long tbar[2], full[NBUF], empty[NBUF];
    __shared__ int fail_p, fail_c;                        // a bounded wait gave up (per role)

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int H = a.H, W = a.W, K = a.K, rt = a.r_th;
    const int nring = 2 * rt + 1;
    const int ty0 = blockIdx.y * TH, tx0 = blockIdx.x * TW;

    float* ring = reinterpret_cast<float*>(smem_raw + 2 * RAW_BUF);       // [nring][RR][P]
    float* Cbuf = ring + (size_t)nring * G::RR * P;                       // [NBUF][RR][P]
    float* Ms = Cbuf + NBUF * G::RR * P;                                  // [RR][P]
    float* gsb = Ms + G::RR * P;                                          // [NBUF][D][GP]
    // raw box of buffer b: [RAW_ROWS][RPT] elements of T
    auto rawbuf = [&](int b) { return reinterpret_cast<T*>(smem_raw + (size_t)b * RAW_BUF); };

    const int reinit = a.sd->reinit;
    // restart: the input is M / (K n_free); read M and fold 1 / (K n_free) into the scale
    const float in_scale = (reinit ? a.inv_uniform : a.sd->inv_Z) * a.out_mult;
    const T* Bin = static_cast<const T*>(a.B_in);
    T* Bout = static_cast<T*>(a.B_out);
    // TMA writes whole boxes into 128-byte aligned buffers
    const bool tma = use_tma && !reinit && (tiled::su32(smem_raw) & 127u) == 0;

    // the map over the region (0 outside the grid)
    for (int q = tid; q < G::RR * RCOLS; q += NT) {
        const int row = q / RCOLS, col = q % RCOLS;
        const int j = ty0 - R + row, i = tx0 - HX + col;
        Ms[row * P + col] = (j >= 0 && j < H && i >= 0 && i < W) ? (float)a.trav[(size_t)j * W + i] : 0.0f;
    }
    if (tid == 0) {
        bar_init(&tbar[0], 1);
        bar_init(&tbar[1], 1);
        for (int b = 0; b < NBUF; ++b) {
            bar_init(&full[b], NP);
            bar_init(&empty[b], NC);
        }
        fail_p = fail_c = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    // Source planes kk0 .. kk_end - 1; plane kk sits in raw buffer (kk - kk0) & 1, its box
    // starting at input column tx0 - HX + ox - xo (xo = 0 on the plain-load path).
    const int kk0 = -rt, kk_end = K + rt;
    auto chan_step = [&](int c) { return c + 1 == K ? 0 : c + 1; };
    const int c0 = ((kk0 % K) + K) % K;
    KahanF acc;

    if (warp < NP / 32) {
        // ------------------------------------------------------------ producers
        const int ptid = tid;
        auto issue = [&](int kk, int c) {                // one thread: TMA of plane kk's box
            const Shift s = a.sh[c];
            const int x = tx0 - HX + s.ox;
            const int b = (kk - kk0) & 1;
            bar_expect(&tbar[b], (uint32_t)(G::RAW_ROWS * RPT * sizeof(T)));
            tma_load(rawbuf(b), &tmap, &tbar[b], x & ~(AL - 1), ty0 - R + s.oy, c);
        };
        auto wait_p = [&](unsigned long long* b, uint32_t parity) {
            if (fail_p) return;
            if (!bar_wait(b, parity)) {
                fail_p = 1;
                atomicOr(&a.sd->status, (unsigned int)LOC_DEV_ERR_TIMEOUT);
            }
        };
        if (tma && ptid == 0) {
            issue(kk0, c0);
            if (kk0 + 1 < kk_end) issue(kk0 + 1, chan_step(c0));
        }
        const float inv_sa = 1.0f / a.sigma_a, inv_sc = 1.0f / a.sigma_c;
        int cur = 0;                                      // ring slot of plane kk: (kk - kk0) mod nring
        int c_cur = c0, c_pre = chan_step(chan_step(c0)); // channels of planes kk and kk + 2
        for (int kk = kk0; kk < kk_end; ++kk) {
            const Shift s = a.sh[c_cur];
            T* rbw = rawbuf((kk - kk0) & 1);
            if (tma) {
                wait_p(&tbar[(kk - kk0) & 1], (uint32_t)(((kk - kk0) >> 1) & 1));
            } else {
                // plain loads of plane kk's box (its buffer was last read two planes ago)
                for (int q = ptid; q < G::RAW_ROWS * RAW_COLS; q += NP) {
                    const int row = q / RAW_COLS, col = q % RAW_COLS;
                    const int gj = ty0 - R + s.oy + row, gi = tx0 - HX + s.ox + col;
                    T v = from_u8<T>(0);
                    if (gj >= 0 && gj < H && gi >= 0 && gi < W) {
                        const size_t o = (size_t)gj * W + gi;
                        v = reinit ? from_u8<T>(a.trav[o]) : Bin[(size_t)c_cur * H * W + o];
                    }
                    rbw[row * RPT + col] = v;
                }
                producers_sync();
            }
            const float fx = s.fx, fy = s.fy, gx0 = 1.0f - fx, gy0 = 1.0f - fy;
            const int xo = tma ? ((tx0 - HX + s.ox) & (AL - 1)) : 0;
            const int o = kk - rt;                        // output channel, once the ring is full
            const bool out = kk - kk0 >= 2 * rt;
            const int b = o % NBUF;
            // C and the stencil of channel o reuse the buffers of channel o - NBUF
            if (out && o >= NBUF) wait_p(&empty[b], (uint32_t)((o / NBUF - 1) & 1));
            float* slot = ring + (size_t)cur * G::RR * P;
            float* Cs = Cbuf + (size_t)b * G::RR * P;
            // ring slots of planes o - rt .. o + rt - 1: (cur + 1 + d) mod nring
            int sl[2 * LOC_MAX_R_THETA];
#pragma unroll
            for (int d = 0; d < 2 * LOC_MAX_R_THETA; ++d) {
                const int v = cur + 1 + d;
                sl[d] = v >= nring ? v - nring : v;
            }
            const T* rb = rbw;
            // S = M * bilinear(raw) into the ring and, once the ring is full, C = theta sum of
            // the ring, 4 cells per item; a producer always owns the same items, so the ring
            // cells it sums are its own writes.  XO = the box's column offset.
            auto fused = [&](auto xo_c) {
                constexpr int XO = decltype(xo_c)::value;
                constexpr int NQ = (G::RR * NG + NP - 1) / NP;
#pragma unroll
                for (int n = 0; n < NQ; ++n) {
                    const int q = ptid + n * NP;
                    if (q >= G::RR * NG) break;
                    const int row = q / NG, g4 = (q % NG) * 4, off = row * P + g4;
                    float r0[RawRow<T>::NV], r1[RawRow<T>::NV], mk[4];
                    RawRow<T>::ld(rb + row * RPT + g4, r0);
                    RawRow<T>::ld(rb + (row + 1) * RPT + g4, r1);
                    ld4(Ms + off, mk);
                    float sv[4];
#pragma unroll
                    for (int x = 0; x < 4; ++x) {
                        const float top = gx0 * r0[XO + x] + fx * r0[XO + x + 1];
                        const float bot = gx0 * r1[XO + x] + fx * r1[XO + x + 1];
                        sv[x] = mk[x] * (gy0 * top + fy * bot);
                    }
                    *reinterpret_cast<float4*>(slot + off) = make_float4(sv[0], sv[1], sv[2], sv[3]);
                    if (out) {
                        float v[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                        for (int d = 0; d < 2 * LOC_MAX_R_THETA; ++d) {
                            if (d < 2 * rt) {
                                const float g = a.gt[d];
                                float x4[4];
                                ld4(ring + (size_t)sl[d] * G::RR * P + off, x4);
#pragma unroll
                                for (int x = 0; x < 4; ++x) v[x] += g * x4[x];
                            }
                        }
                        const float g = a.gt[2 * rt];     // the newest plane, o + rt
#pragma unroll
                        for (int x = 0; x < 4; ++x) v[x] += g * sv[x];
                        *reinterpret_cast<float4*>(Cs + off) = make_float4(v[0], v[1], v[2], v[3]);
                    }
                }
            };
            switch (xo) {
                case 0: fused(IC<0>{}); break;
                case 1: fused(IC<1>{}); break;
                case 2: fused(IC<2>{}); break;
                case 3: fused(IC<3>{}); break;
                default:
                    if constexpr (AL == 8) {
                        switch (xo) {
                            case 4: fused(IC<4>{}); break;
                            case 5: fused(IC<5>{}); break;
                            case 6: fused(IC<6>{}); break;
                            default: fused(IC<7>{}); break;
                        }
                    }
            }
            if (out) {
                // channel o's x/y stencil (unnormalised), row-major with pitch GP
                const float phi = a.phi0 + a.dphi * (float)o;
                float sp, cp;
                sincosf(phi, &sp, &cp);
                float* gs = gsb + b * G::D * G::GP;
                // taps spread over all producer warps (q = 2 ptid, 2 ptid + 1 ...)
                constexpr int NTAP = G::D * G::GP;
                constexpr int SPREAD = NTAP * 2 <= NP ? 2 : 1;
                for (int q0 = ptid; q0 < NTAP * SPREAD; q0 += NP) {
                    if (q0 % SPREAD) continue;
                    const int q = q0 / SPREAD;
                    const int dj = q / G::GP, di = q % G::GP;
                    float w = 0.0f;
                    if (di < G::D) {
                        const float fdj = (float)(dj - R), fdi = (float)(di - R);
                        const float along = (fdi * cp + fdj * sp) * inv_sa;
                        const float across = (fdj * cp - fdi * sp) * inv_sc;
                        w = expf(-0.5f * (along * along + across * across));
                    }
                    gs[q] = w;
                }
            }
            producers_sync();                             // every producer has read the raw box
            if (tma && ptid == 0 && kk + 2 < kk_end) issue(kk + 2, c_pre);   // into the box just read
            if (out) bar_arrive(&full[b]);                // C and the stencil of channel o are ready
            cur = cur + 1 == nring ? 0 : cur + 1;
            c_cur = chan_step(c_cur);
            c_pre = chan_step(c_pre);
        }
    } else {
        // ------------------------------------------------------------ consumers
        // this thread's block: output rows oy0 .. oy0+BY-1, columns ox0 .. ox0+3 of the tile
        const int cw = warp - NP / 32;
        const int lx = lane & 7, ly = lane >> 3;
        const int oy0 = 4 * BY * cw + BY * ly, ox0 = 4 * lx;
        bool interior = true;
        for (int r = 0; r < G::NR; ++r)
            for (int cc = HX - R; cc < HX + 4 + R; ++cc) interior &= Ms[(oy0 + r) * P + ox0 + cc] > 0.0f;
        uint32_t free_bits = 0;                           // centres of this block that are free
#pragma unroll
        for (int y = 0; y < BY; ++y)
#pragma unroll
            for (int x = 0; x < 4; ++x)
                if (Ms[(oy0 + y + R) * P + HX + ox0 + x] > 0.0f) free_bits |= 1u << (4 * y + x);
        // per warp: every lane interior (G_k is the stencil sum) / some lane with a free cell
        const bool warp_interior = __all_sync(0xffffffffu, interior);
        const bool warp_any_free = __any_sync(0xffffffffu, free_bits != 0);
        float res[BY][4];                                 // BF16 residuals of the block's cells
#pragma unroll
        for (int y = 0; y < BY; ++y)
#pragma unroll
            for (int x = 0; x < 4; ++x) res[y][x] = 0.0f;
        for (int o = 0; o < K; ++o) {
            const int b = o % NBUF;
            if (!fail_c && !bar_wait(&full[b], (uint32_t)((o / NBUF) & 1))) {
                fail_c = 1;
                atomicOr(&a.sd->status, (unsigned int)LOC_DEV_ERR_TIMEOUT);
            }
            const float* Cs = Cbuf + (size_t)b * G::RR * P;
            const float* gs = gsb + b * G::D * G::GP;
            float part = 0.0f;
            T* oplane = Bout + (size_t)o * H * W;
            if (warp_any_free) {
                float t[BY][4], gm[BY][4];
#pragma unroll
                for (int y = 0; y < BY; ++y)
#pragma unroll
                    for (int x = 0; x < 4; ++x) t[y][x] = gm[y][x] = 0.0f;
                const int base = oy0 * P + ox0;
                if (warp_interior) {
                    stencil_block<R, false>(Cs + base, Ms + base, gs, t, gm);
                    // every map cell under the window is 1: G_k is the stencil's sum, taken in
                    // the row-major order of the FMAs it replaces (fma(w, 1, s) = s + w)
                    float sum = 0.0f;
#pragma unroll
                    for (int dj = 0; dj < G::D; ++dj)
#pragma unroll
                        for (int di = 0; di < G::D; ++di) sum = fmaf(gs[dj * G::GP + di], 1.0f, sum);
#pragma unroll
                    for (int y = 0; y < BY; ++y)
#pragma unroll
                        for (int x = 0; x < 4; ++x) gm[y][x] = sum;
                } else {
                    stencil_block<R, true>(Cs + base, Ms + base, gs, t, gm);
                }
                bar_arrive(&empty[b]);                    // C and the stencil of channel o are read
#pragma unroll
                for (int y = 0; y < BY; ++y) {
                    const int gj = ty0 + oy0 + y, gi = tx0 + ox0;
                    if (gj >= H) break;
                    T ov[4];
                    const size_t off = (size_t)gj * W + gi;
#pragma unroll
                    for (int x = 0; x < 4; ++x) {
                        // gm >= 1 on a free cell (its own tap is exp(0))
                        const float v = (free_bits >> (4 * y + x)) & 1u ? __fdividef(t[y][x], gm[y][x]) * in_scale : 0.0f;
                        ov[x] = round_out<T>(v, res[y][x]);
                    }
                    if ((W & 3) == 0 && gi + 3 < W) {
                        Vec4<T>::st(oplane + off, ov);
#pragma unroll
                        for (int x = 0; x < 4; ++x) part += to_f<T>(ov[x]);
                    } else {
#pragma unroll
                        for (int x = 0; x < 4; ++x)
                            if (gi + x < W) {
                                oplane[off + x] = ov[x];
                                part += to_f<T>(ov[x]);
                            }
                    }
                }
            } else {
                bar_arrive(&empty[b]);
                const T zero = T(0.0f);
#pragma unroll
                for (int y = 0; y < BY; ++y) {
                    const int gj = ty0 + oy0 + y, gi = tx0 + ox0;
                    if (gj >= H) break;
#pragma unroll
                    for (int x = 0; x < 4; ++x)
                        if (gi + x < W) oplane[(size_t)gj * W + gi + x] = zero;
                }
            }
            acc.add(part);
        }
    }
    __syncthreads();

    const double bt = block_sum<NT>(acc.value(), red);
    const unsigned int nblocks = gridDim.x * gridDim.y;
    SessionDev* sd = a.sd;
    const double log_mult = a.log_out_mult;
    finish_sum<NT>(bt, a.partials, &sd->counter, nblocks, red, [sd, log_mult](double Z) {
        sd->n_prop += 1;
        if (Z > 0.0 && isfinite(Z)) {
            sd->Z = Z;
            sd->inv_Z = (float)(1.0 / Z);
            sd->logscale += log(Z) - log_mult;
            sd->reinit = 0;
        } else {
            if (!isfinite(Z)) sd->status |= LOC_DEV_ERR_NONFINITE_Z;
            sd->Z = 1.0;
            sd->inv_Z = 1.0f;
            sd->reinit = 1;
            sd->n_reinit += 1;
        }
    });
}

template <typename T, int R>
cudaError_t launch_r(const StepArgs& a, const void* tmap, cudaStream_t st) {
    const size_t smem = aniso_smem_bytes<T, R>(a.r_th);
    static bool attr_set[64] = {};                // per device: the largest size any session asks for
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || !attr_set[dev]) {
        const cudaError_t e = cudaFuncSetAttribute(step_aniso_kernel<T, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)aniso_smem_bytes<T, R>(LOC_MAX_R_THETA));
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) attr_set[dev] = true;
    }
    CUtensorMap tm;
    memset(&tm, 0, sizeof(tm));
    if (tmap) memcpy(&tm, tmap, sizeof(tm));
    dim3 grid((a.W + TW - 1) / TW, (a.H + TH - 1) / TH);
    step_aniso_kernel<T, R><<<grid, NT, smem, st>>>(a, tm, tmap ? 1 : 0);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_t(const StepArgs& a, const void* tmap, cudaStream_t st) {
    switch (a.r_xy) {
        case 0: return launch_r<T, 0>(a, tmap, st);
        case 1: return launch_r<T, 1>(a, tmap, st);
        case 2: return launch_r<T, 2>(a, tmap, st);
        case 3: return launch_r<T, 3>(a, tmap, st);
        case 4: return launch_r<T, 4>(a, tmap, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

bool aniso_tma_eligible(int W, int storage) {
    // the row pitch of a belief plane must be a multiple of 16 bytes
    return storage == LOC_F32 ? W % 4 == 0 : W % 8 == 0;
}

cudaError_t make_aniso_tmap(void* tmap_out, const void* B, int storage, int H, int W, int K, int r_xy) {
    if (!aniso_tma_eligible(W, storage) || r_xy < 0 || r_xy > LOC_MAX_R_XY) return cudaErrorInvalidValue;
    const int bw = storage == LOC_F32 ? raw_pitch<float>() : raw_pitch<__half>();
    return make_box_tmap(tmap_out, B, storage, H, W, K, bw, TH + 2 * r_xy + 1);
}

cudaError_t launch_step_aniso(const StepArgs& a, const void* tmap, int storage, cudaStream_t st) {
    static_assert(LOC_MAX_R_XY <= HX, "the region's left margin must cover the x/y radius");
    static_assert(NC == 4 * 32 && TH == 4 * 4 * BY && TW == 32 && NP % 32 == 0,
                  "4 consumer warps of 8 x 4 lanes cover the tile; whole producer warps");
    static_assert(RAW_COLS + 3 <= 44 && RAW_COLS + 7 <= 48, "the box covers 41 columns after the x rounding");
    if (a.r_xy < 0 || a.r_xy > LOC_MAX_R_XY || a.r_th < 0 || a.r_th > LOC_MAX_R_THETA ||
        !(a.sigma_a > 0.0f) || !(a.sigma_c > 0.0f))
        return cudaErrorInvalidValue;
    switch (storage) {
        case LOC_F32: return launch_t<float>(a, tmap, st);
        case LOC_BF16: return launch_t<__nv_bfloat16>(a, tmap, st);
        case LOC_F16: return launch_t<__half>(a, tmap, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace loc
