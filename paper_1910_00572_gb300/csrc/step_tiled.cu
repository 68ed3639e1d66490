// Tiled fused propagation kernel for the default motion kernel (x/y radius 2, theta radius 3):
// Algorithm 1's propagation for all K channels plus the Eq. 9 normaliser in one pass over HBM.
//
// One CTA owns a TH x 64 output tile and streams the planes p = 0 .. K+5:
//   * raw tile of X_{t-1}[p] around the tile, shifted by the plane's integer source offset,
//     arrives by TMA (cp.async.bulk.tensor.3d, zero fill off the grid) NSTAGE-1 planes ahead
//     into a ring of stages guarded by mbarriers;
//   * S-pass: S = M * bilinear(raw) over the (TH+4) x 68 halo region (Eq. 3, Algorithm 1's first mask);
//   * X-pass: X = x-blur(S) over (TH+4) x 64 (Eq. 7, separable for the isotropic kernel);
//   * P-pass: each thread owns 2 x MR output cells, applies the y-blur and pushes the result
//     into a 7-deep register ring over theta; once the ring holds planes p-6 .. p it writes
//     channel p-3 = corr * scale * sum_d gt[d] P[p-3+d] (theta blur, Algorithm 1's mask + edge correction,
//     Eq. 8) and adds the stored (rounded) values to its FP32 partial.
// The circular theta blur needs planes 0..5 again at the end: the P-pass keeps them in
// shared memory (planes p = K .. K+5 read them back), so every input plane is read from HBM
// once.  CTA partials are combined in FP64 by the last CTA (Z, log-scale).
//
// Tile configurations (Cfg1..Cfg16) trade halo overhead against the number of resident CTAs
// and how the passes are spread over warps; the session picks one per grid shape.
#include <type_traits>

#include "tiled_pairs.cuh"

namespace loc {
namespace {

using namespace tiled;

// The last CTA's update of the session scalars from the new normaliser Z (Eq. 9): Z, 1/Z and
// the log-scale, or the uniform restart when no mass is left.
__device__ __forceinline__ void finish_step(SessionDev* sd, double Z, double log_mult) {
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
}

template <typename T, typename C>
__global__ void __launch_bounds__(C::NT, C::MINB) step_tiled_kernel(const __grid_constant__ FastArgs a) {
    constexpr int NT = C::NT, NSTAGE = C::NSTAGE;
    constexpr bool PAIRS = C::PAIRS;
    using SM = std::conditional_t<PAIRS, pairs::PSmem<T, C>, std::conditional_t<C::PIPE, SmemPipe<T, C>, Smem<T, C>>>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // the dynamic region is only guaranteed 16-byte aligned: round up to 128 bytes
    const uint32_t base = su32(smem_raw);
    SM& sm = *reinterpret_cast<SM*>(smem_raw + (((base + 127u) & ~127u) - base));
    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int s = 0; s < NSTAGE; ++s) bar_init(&sm.bar[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    TileJob j;
    j.tmap = &a.tmap;
    j.sh = a.sh;
    j.o.B_out = a.B_out;
    j.o.H = a.H;
    j.o.W = a.W;
    j.o.K = a.K;
    j.trav = a.trav;
    j.corr = a.corr;
    j.gt = a.gt;
    j.reinit = a.sd->reinit;
    // restart: the input is M / (K n_free); read M and fold 1 / (K n_free) into the scale
    j.in_scale = (j.reinit ? a.inv_uniform : a.sd->inv_Z) * a.out_mult;
    j.g0 = a.g0;
    j.g1 = a.g1;
    j.g2 = a.g2;
    j.ty0 = blockIdx.y * C::TH;
    j.tx0 = blockIdx.x * TW;
    std::conditional_t<PAIRS, KahanF, KahanF2> acc;
    int p_stop = 0, next_issue = 0;
    bool ok;
    if constexpr (PAIRS) ok = pairs::run_tile<T, C>(sm, j, 0u, acc, p_stop, next_issue);
    else if constexpr (C::PIPE) ok = run_tile_pipe<T, C>(sm, j, 0u, acc, p_stop, next_issue);
    else ok = run_tile<T, C>(sm, j, 0u, acc, p_stop, next_issue);
    if (!ok) {
        // a TMA wait gave up: report it, let the copies still in flight land (bounded), and
        // leave without contributing a partial (the host sees the flag and fails the handle)
        if (tid == 0) {
            atomicOr(&a.sd->status, LOC_DEV_ERR_TIMEOUT);
            for (int q = p_stop; q < next_issue; ++q) bar_wait(&sm.bar[q % NSTAGE], (uint32_t)((q / NSTAGE) & 1));
        }
        __syncthreads();
        return;
    }
    const double bt = block_sum<NT>(acc.value(), sm.red);
    SessionDev* sd = a.sd;
    const double log_mult = a.log_out_mult;
    finish_sum<NT>(bt, a.partials, &sd->counter, gridDim.x * gridDim.y, sm.red,
                   [sd, log_mult](double Z) { finish_step(sd, Z, log_mult); });
}

// ---------------------------------------------------------------------------------------------
// Warp-specialised variant.  Producer warps run the S-pass and X-pass of plane p+1 while
// consumer warps run the P-pass of plane p; the X plane is double-buffered between them.
// Hand-offs use mbarriers with bounded waits (FULL[b]: the X-pass threads arrive after writing
// X[b]; EMPTY[b]: consumers arrive after reading it); producers synchronise among themselves
// with a named barrier that every producer thread reaches on every plane.  With SPLIT the
// producers are two groups: S warps run the S-pass of plane p while X warps run the X-pass of
// plane p - 1, between the same two producer barriers.  The consumers, which wait on the
// producers, also keep the running argmax of the values they store; the last CTA combines it
// with the normaliser, so a pose read after the step needs no pass over the tensor.

__device__ __forceinline__ void bar_arrive(unsigned long long* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}
template <int NP>
__device__ __forceinline__ void producers_sync() {       // named barrier 1, producer threads only
    asm volatile("bar.sync 1, %0;" ::"n"(NP) : "memory");
}
template <int NS>
__device__ __forceinline__ void s_threads_sync() {       // named barrier 2, S threads of a split
    asm volatile("bar.sync 2, %0;" ::"n"(NS) : "memory");
}

// TH tile rows, SR S-pass rows per item, XW X-pass columns per item, NSTAGE raw stages, MINB
// CTAs per SM asked of the compiler, NP / NC producer / consumer threads, MR consumer rows per
// thread (2 columns each; 0: TH * 64 / (2 NC)).  The consumers cover CR = MR * NC / 32 >= TH
// rows; rows TH .. CR-1 are computed from zero X rows and never stored, so TH need not be a
// multiple of MR.  SPLIT divides the producers into S warps (the first NS threads) and X warps
// (the other NX): the S-pass of plane p and the X-pass of plane p - 1 then run side by side
// between two producer barriers instead of one after the other.
template <int TH_, int SR_, int XW_, int NSTAGE_, int MINB_, int NP_ = 128, int NC_ = 128, int MR_ = 0,
          bool SPLIT_ = false>
struct WsCfg {
    static constexpr int TH = TH_, SR = SR_, XW = XW_, NSTAGE = NSTAGE_, MINB = MINB_;
    static constexpr int NP = NP_, NC = NC_, NT = NP + NC;
    static constexpr bool SPLIT = SPLIT_;
    static_assert(NP % 32 == 0 && NC % 32 == 0, "whole producer and consumer warps");
    static constexpr int MR = MR_ > 0 ? MR_ : TH * TW / (2 * NC);   // consumer rows per thread
    static constexpr int CR = MR * (NC / 32);                         // rows the consumers cover
    static constexpr int XR = TH + 2 * R;                             // S and X rows computed
    static constexpr int XRC = CR + 2 * R;                            // X rows the consumers read
    static constexpr int RAW_H = XR + 1;
    static constexpr int S_ITEMS = (72 / 4) * (XR / SR), X_ITEMS = (TW / XW) * XR;
    static constexpr int NS = SPLIT ? (S_ITEMS + 31) / 32 * 32 : NP;  // threads of the S-pass
    static constexpr int NX = SPLIT ? NP - NS : NP;                   // threads of the X-pass
    static_assert(XR % SR == 0, "S-pass row groups must tile the halo rows");
    static_assert(S_ITEMS <= NS, "one S-pass item per S thread");
    static_assert(X_ITEMS <= NX, "one X-pass item per X thread");
    static_assert(CR >= TH && CR - MR < TH, "consumer tiling: every consumer warp has a row in the tile");
};

template <typename T, typename C>
struct SmemWS {
    T raw[C::NSTAGE][raw_stride<T, C>()];
    float S[2][C::XR][SW];                   // S of planes p and p + 1 (the X-pass of p overlaps)
    float X[2][C::XRC][XW_PITCH];            // rows XR .. XRC-1 stay zero
    float wrap[NWRAP][C::CR][TW];
    float mk[C::XR][MW];
    unsigned long long tma[C::NSTAGE];
    unsigned long long full[2], empty[2];
    // failure flags (a bounded wait gave up): producers set fail_a (TMA) and fail_b (EMPTY),
    // consumers fail_c.  A set flag only skips work and further waits; no thread leaves its
    // loop early, so every producer reaches every named barrier.
    int fail_a, fail_b, fail_c;
    double red[C::NT / 32];
};

template <typename T, typename C>
__global__ void __launch_bounds__(C::NT, C::MINB) step_ws_kernel(const __grid_constant__ FastArgs a) {
    constexpr int NT = C::NT, NP = C::NP, TH = C::TH, MR = C::MR, NSTAGE = C::NSTAGE, XR = C::XR;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const uint32_t base = su32(smem_raw);
    SmemWS<T, C>& sm = *reinterpret_cast<SmemWS<T, C>*>(smem_raw + (((base + 127u) & ~127u) - base));
    const int tid = threadIdx.x;
    const int H = a.H, W = a.W, K = a.K;
    const int ty0 = blockIdx.y * TH, tx0 = blockIdx.x * TW;
    const int reinit = a.sd->reinit;
    const float in_scale = (reinit ? a.inv_uniform : a.sd->inv_Z) * a.out_mult;
    constexpr uint32_t kBoxBytes = C::RAW_H * BW * sizeof(T);

    for (int q = tid; q < XR * MW; q += NT) {
        const int y = q / MW, c = q % MW;
        const int gy = ty0 - R + y, gx = tx0 - R + c;
        sm.mk[y][c] = (gy >= 0 && gy < H && gx >= 0 && gx < W && a.trav[(size_t)gy * W + gx]) ? 1.0f : 0.0f;
    }
    if constexpr (C::XRC > XR) {
        for (int q = tid; q < 2 * (C::XRC - XR) * XW_PITCH; q += NT) {
            const int b = q / ((C::XRC - XR) * XW_PITCH), r = q % ((C::XRC - XR) * XW_PITCH);
            sm.X[b][XR + r / XW_PITCH][r % XW_PITCH] = 0.0f;
        }
    }
    if (tid == 0) {
        for (int s = 0; s < NSTAGE; ++s) bar_init(&sm.tma[s], 1);
        for (int b = 0; b < 2; ++b) {
            bar_init(&sm.full[b], C::NX);
            bar_init(&sm.empty[b], C::NC);
        }
        sm.fail_a = sm.fail_b = sm.fail_c = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();

    KahanF2 acc;
    ArgBest am;                             // consumers: the argmax of the values they store
    int waited = 0, next_issue = 0;         // producer: planes [waited, next_issue) maybe in flight
    if (tid < NP) {
        // ------------------------------------------------------------------ producers
        const int t = tid;
        // items: in a split, the S threads are the first NS and the X threads the rest
        const SItem si = s_item<C>(t);
        const XItem xi = x_item<C>(C::SPLIT ? t - C::NS : t);
        auto issue = [&](int q) {
            const Shift s = a.sh[q];
            int x_al, xo;
            box_x<T>(tx0, s, x_al, xo);
            bar_expect(&sm.tma[q % NSTAGE], kBoxBytes);
            tma_load(&sm.raw[q % NSTAGE][0], &a.tmap, &sm.tma[q % NSTAGE], x_al, ty0 - R + s.oy, q);
        };
        if (!reinit) {
            next_issue = NSTAGE < K ? NSTAGE : K;
            if (t == 0)
                for (int q = 0; q < next_issue; ++q) issue(q);
        }
        if constexpr (C::SPLIT) {
            // S threads take plane p, X threads plane p - 1.  S of plane p goes to S[p & 1], which
            // the X-pass of plane p - 2 finished reading before the previous producer barrier;
            // the X-pass of plane p - 1 reads S[(p - 1) & 1], complete since that barrier.
            const bool s_role = t < C::NS;
            for (int p = 0; p <= K; ++p) {
                if (s_role) {
                    if (p < K) {
                        const int stage = p % NSTAGE;
                        const Shift s = a.sh[p];
                        int x_al, xo;
                        box_x<T>(tx0, s, x_al, xo);
                        if (reinit) {
                            const int y0 = ty0 - R + s.oy;
                            for (int q = t; q < C::RAW_H * BW; q += C::NS) {
                                const int y = q / BW, c = q % BW;
                                const int gy = y0 + y, gx = x_al + c;
                                float v = 0.0f;
                                if (gy >= 0 && gy < H && gx >= 0 && gx < W) v = (float)a.trav[(size_t)gy * W + gx];
                                sm.raw[stage][y * BW + c] = T(v);
                            }
                            s_threads_sync<C::NS>();
                        } else if (!sm.fail_a) {
                            if (bar_wait(&sm.tma[stage], (uint32_t)((p / NSTAGE) & 1))) waited = p + 1;
                            else sm.fail_a = 1;
                        }
                        if (!sm.fail_a) s_pass_any<T, C>(sm.raw[stage], &sm.mk[0][0], &sm.S[p & 1][0][0], si, xo, s.fx, s.fy);
                    }
                } else if (p >= 1) {
                    const int q = p - 1, b = q & 1;
                    if (q >= 2 && !sm.fail_b && !bar_wait(&sm.empty[b], (uint32_t)(((q - 2) >> 1) & 1))) sm.fail_b = 1;
                    if (!(sm.fail_a | sm.fail_b)) x_pass<C>(&sm.S[b][0][0], &sm.X[b][0][0], xi, a.g0, a.g1, a.g2);
                    bar_arrive(&sm.full[b]);             // X[b] of plane p - 1 is ready
                }
                producers_sync<NP>();
                if (p < K && !reinit && p + NSTAGE < K && !sm.fail_a) {
                    if (t == 0) {
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        issue(p + NSTAGE);
                    }
                    next_issue = p + NSTAGE + 1;
                }
            }
        } else for (int p = 0; p < K; ++p) {
            const int stage = p % NSTAGE;
            float (*S)[SW] = sm.S[p & 1];
            const Shift s = a.sh[p];
            int x_al, xo;
            box_x<T>(tx0, s, x_al, xo);
            if (reinit) {
                const int y0 = ty0 - R + s.oy;
                for (int q = t; q < C::RAW_H * BW; q += NP) {
                    const int y = q / BW, c = q % BW;
                    const int gy = y0 + y, gx = x_al + c;
                    float v = 0.0f;
                    if (gy >= 0 && gy < H && gx >= 0 && gx < W) v = (float)a.trav[(size_t)gy * W + gx];
                    sm.raw[stage][y * BW + c] = T(v);
                }
                producers_sync<NP>();
            } else if (!sm.fail_a) {
                if (bar_wait(&sm.tma[stage], (uint32_t)((p / NSTAGE) & 1))) waited = p + 1;
                else sm.fail_a = 1;
            }
            if (!sm.fail_a) s_pass_any<T, C>(sm.raw[stage], &sm.mk[0][0], &S[0][0], si, xo, s.fx, s.fy);
            // S of plane p complete and the raw stage free; every producer has also finished the
            // X-pass of plane p - 1, so S of plane p + 1 (the other buffer's next use) may be written
            producers_sync<NP>();
            if (!reinit && p + NSTAGE < K && !sm.fail_a) {
                if (t == 0) {
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    issue(p + NSTAGE);
                }
                next_issue = p + NSTAGE + 1;
            }
            const int b = p & 1;
            if (p >= 2 && !sm.fail_b && !bar_wait(&sm.empty[b], (uint32_t)(((p - 2) >> 1) & 1))) sm.fail_b = 1;
            if (!(sm.fail_a | sm.fail_b)) x_pass<C>(&S[0][0], &sm.X[b][0][0], xi, a.g0, a.g1, a.g2);
            bar_arrive(&sm.full[b]);                 // X[b] of plane p is ready
        }
    } else {
        // ------------------------------------------------------------------ consumers
        const int t = tid - NP;
        const int cp = t % 32, rg = t / 32;
        const int r0 = MR * rg, gxp = tx0 + 2 * cp;
        f2 cs[MR];
#pragma unroll
        for (int rr = 0; rr < MR; ++rr) {
            const int gy = ty0 + r0 + rr;
            float c0 = 0.0f, c1 = 0.0f;
            if (gy < H && gxp < W && r0 + rr < TH) {
                c0 = a.corr[(size_t)gy * W + gxp] * in_scale;
                c1 = a.corr[(size_t)gy * W + gxp + 1] * in_scale;
            }
            cs[rr] = pk(c0, c1);
        }
        Taps2 tp;
        tp.g0 = pk(a.g0, a.g0);
        tp.g1 = pk(a.g1, a.g1);
        tp.g2 = pk(a.g2, a.g2);
#pragma unroll
        for (int d = 0; d < RING; ++d) tp.gt[d] = pk(a.gt[d], a.gt[d]);
        f2 ring[RING][MR], res[MR];
#pragma unroll
        for (int d = 0; d < RING; ++d)
#pragma unroll
            for (int k = 0; k < MR; ++k) ring[d][k] = 0ull;
#pragma unroll
        for (int k = 0; k < MR; ++k) res[k] = 0ull;
        TileOut o;
        o.B_out = a.B_out;
        o.H = H;
        o.W = W;
        o.K = K;
        const PCtx<T> pc = p_ctx<T, C>(o, r0, ty0, gxp);
        for (int p = 0, ph = 0; p < K + NWRAP; ++p, ph = ph == RING - 1 ? 0 : ph + 1) {
            const int b = p & 1;
            if (p < K && !bar_wait(&sm.full[b], (uint32_t)((p >> 1) & 1))) {
                sm.fail_c = 1;
                break;
            }
            switch (ph) {
                case 0: p_pass<T, C, 0, true>(sm.X[b], sm.wrap, pc, K, tp, ring, cs, res, p, r0, cp, acc, &am); break;
                case 1: p_pass<T, C, 1, true>(sm.X[b], sm.wrap, pc, K, tp, ring, cs, res, p, r0, cp, acc, &am); break;
                case 2: p_pass<T, C, 2, true>(sm.X[b], sm.wrap, pc, K, tp, ring, cs, res, p, r0, cp, acc, &am); break;
                case 3: p_pass<T, C, 3, true>(sm.X[b], sm.wrap, pc, K, tp, ring, cs, res, p, r0, cp, acc, &am); break;
                case 4: p_pass<T, C, 4, true>(sm.X[b], sm.wrap, pc, K, tp, ring, cs, res, p, r0, cp, acc, &am); break;
                case 5: p_pass<T, C, 5, true>(sm.X[b], sm.wrap, pc, K, tp, ring, cs, res, p, r0, cp, acc, &am); break;
                default: p_pass<T, C, 6, true>(sm.X[b], sm.wrap, pc, K, tp, ring, cs, res, p, r0, cp, acc, &am); break;
            }
            if (p + 2 < K) bar_arrive(&sm.empty[b]);  // a producer waits for this release
        }
    }
    __syncthreads();
    if (sm.fail_a | sm.fail_b | sm.fail_c) {
        if (tid == 0) {
            atomicOr(&a.sd->status, LOC_DEV_ERR_TIMEOUT);
            for (int q = waited; q < next_issue; ++q) bar_wait(&sm.tma[q % NSTAGE], (uint32_t)((q / NSTAGE) & 1));
        }
        __syncthreads();
        return;
    }
    const double bt = block_sum<NT>(acc.value(), sm.red);
    SessionDev* sd = a.sd;
    const double log_mult = a.log_out_mult;
    finish_sum_am<NT>(bt, am, a.partials, a.am_pv, a.am_pi, &sd->counter, gridDim.x * gridDim.y, sm.red, a.am_idx,
                      a.am_val, [sd, log_mult](double Z) { finish_step(sd, Z, log_mult); });
}

// The tile configurations.  1: 32-row tiles (large grids); 2: 16-row tiles with 2-row
// P-pass items (256 threads); 3: 16-row tiles with 4-row P-pass items (128 threads).
using Cfg1 = Cfg<32, 4, 3, 16, 3, 2>;
using Cfg2 = Cfg<16, 2, 2, 8, 3, 3>;
using Cfg3 = Cfg<16, 4, 4, 16, 3, 4>;
using Cfg4 = Cfg<16, 1, 2, 8, 3, 2>;
using Cfg5 = Cfg<32, 2, 3, 16, 3, 1>;
using Cfg6 = WsCfg<16, 4, 16, 3, 2>;   // warp-specialised, 16-row tiles
using Cfg7 = WsCfg<8, 2, 8, 3, 4>;     // warp-specialised, 8-row tiles
// Paired-column passes (tiled_pairs.cuh): 8: 16-row tiles, 128 threads; 9: 16-row tiles, 256
// threads; 10: 32-row tiles, 256 threads, 2 raw stages; 11: 8-row tiles, 128 threads;
// 12: 16-row tiles, 128 threads, 2 raw stages, 4 CTAs per SM.
using Cfg8 = pairs::PCfg<16, 4, 2, 8, 3, 3>;
using Cfg9 = pairs::PCfg<16, 2, 2, 4, 3, 2>;
using Cfg10 = pairs::PCfg<32, 4, 2, 8, 2, 2>;
using Cfg11 = pairs::PCfg<8, 2, 2, 8, 3, 4>;
using Cfg12 = pairs::PCfg<16, 4, 2, 8, 2, 4>;
// 13: warp-specialised 14-row tiles (the consumers cover 16 rows, 14 stored); 14-16: split
// producers (S warps beside X warps): 14: 16-row tiles, 96 + 96 producer threads; 15: 14-row
// tiles, 64 + 96; 16: 28-row tiles, one CTA of 16 warps per SM (160 + 128 producer threads,
// 224 consumer threads).
using Cfg13 = WsCfg<14, 3, 16, 3, 2, 128, 128, 4>;
using Cfg14 = WsCfg<16, 4, 16, 3, 2, 192, 128, 0, true>;
using Cfg15 = WsCfg<14, 6, 16, 3, 2, 160, 128, 4, true>;
using Cfg16 = WsCfg<28, 4, 16, 3, 1, 288, 224, 4, true>;
// 17, 18: configurations 3 and 2 as a software pipeline over the planes (run_tile_pipe: one
// CTA barrier per plane, S and X double-buffered).
using Cfg17 = Cfg<16, 4, 4, 16, 3, 3, true>;
using Cfg18 = Cfg<16, 2, 2, 8, 3, 3, true>;

template <typename T, typename C> size_t smem_bytes() {
    using SM = std::conditional_t<C::PAIRS, pairs::PSmem<T, C>, std::conditional_t<C::PIPE, SmemPipe<T, C>, Smem<T, C>>>;
    return sizeof(SM) + 128;
}

// Launch with the dynamic shared memory size; the attribute is set once per device.
template <typename T, typename C>
cudaError_t launch_typed(const FastArgs& a, dim3 grid, cudaStream_t st) {
    static bool attr_set[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    const size_t sb = smem_bytes<T, C>();
    if (dev < 0 || dev >= 64 || !attr_set[dev]) {
        cudaError_t e = cudaFuncSetAttribute(step_tiled_kernel<T, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sb);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) attr_set[dev] = true;
    }
    step_tiled_kernel<T, C><<<grid, C::NT, sb, st>>>(a);
    return cudaSuccess;
}

template <typename T, typename C>
cudaError_t launch_ws(const FastArgs& a, dim3 grid, cudaStream_t st) {
    static bool attr_set[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    const size_t sb = sizeof(SmemWS<T, C>) + 128;
    if (dev < 0 || dev >= 64 || !attr_set[dev]) {
        cudaError_t e = cudaFuncSetAttribute(step_ws_kernel<T, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sb);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) attr_set[dev] = true;
    }
    step_ws_kernel<T, C><<<grid, C::NT, sb, st>>>(a);
    return cudaSuccess;
}

template <typename T>
cudaError_t launch_cfg(int cfg, const FastArgs& a, int W, int H, cudaStream_t st) {
    switch (cfg) {
        case 1: return launch_typed<T, Cfg1>(a, dim3((W + TW - 1) / TW, (H + Cfg1::TH - 1) / Cfg1::TH), st);
        case 2: return launch_typed<T, Cfg2>(a, dim3((W + TW - 1) / TW, (H + Cfg2::TH - 1) / Cfg2::TH), st);
        case 3: return launch_typed<T, Cfg3>(a, dim3((W + TW - 1) / TW, (H + Cfg3::TH - 1) / Cfg3::TH), st);
        case 4: return launch_typed<T, Cfg4>(a, dim3((W + TW - 1) / TW, (H + Cfg4::TH - 1) / Cfg4::TH), st);
        case 5: return launch_typed<T, Cfg5>(a, dim3((W + TW - 1) / TW, (H + Cfg5::TH - 1) / Cfg5::TH), st);
        case 6: return launch_ws<T, Cfg6>(a, dim3((W + TW - 1) / TW, (H + Cfg6::TH - 1) / Cfg6::TH), st);
        case 7: return launch_ws<T, Cfg7>(a, dim3((W + TW - 1) / TW, (H + Cfg7::TH - 1) / Cfg7::TH), st);
        case 8: return launch_typed<T, Cfg8>(a, dim3((W + TW - 1) / TW, (H + Cfg8::TH - 1) / Cfg8::TH), st);
        case 9: return launch_typed<T, Cfg9>(a, dim3((W + TW - 1) / TW, (H + Cfg9::TH - 1) / Cfg9::TH), st);
        case 10: return launch_typed<T, Cfg10>(a, dim3((W + TW - 1) / TW, (H + Cfg10::TH - 1) / Cfg10::TH), st);
        case 11: return launch_typed<T, Cfg11>(a, dim3((W + TW - 1) / TW, (H + Cfg11::TH - 1) / Cfg11::TH), st);
        case 12: return launch_typed<T, Cfg12>(a, dim3((W + TW - 1) / TW, (H + Cfg12::TH - 1) / Cfg12::TH), st);
        case 13: return launch_ws<T, Cfg13>(a, dim3((W + TW - 1) / TW, (H + Cfg13::TH - 1) / Cfg13::TH), st);
        case 14: return launch_ws<T, Cfg14>(a, dim3((W + TW - 1) / TW, (H + Cfg14::TH - 1) / Cfg14::TH), st);
        case 15: return launch_ws<T, Cfg15>(a, dim3((W + TW - 1) / TW, (H + Cfg15::TH - 1) / Cfg15::TH), st);
        case 16: return launch_ws<T, Cfg16>(a, dim3((W + TW - 1) / TW, (H + Cfg16::TH - 1) / Cfg16::TH), st);
        case 17: return launch_typed<T, Cfg17>(a, dim3((W + TW - 1) / TW, (H + Cfg17::TH - 1) / Cfg17::TH), st);
        case 18: return launch_typed<T, Cfg18>(a, dim3((W + TW - 1) / TW, (H + Cfg18::TH - 1) / Cfg18::TH), st);
        default: return cudaErrorInvalidValue;
    }
}

int cfg_tile_rows(int cfg) {
    switch (cfg) {
        case 1: return Cfg1::TH;
        case 2: return Cfg2::TH;
        case 3: return Cfg3::TH;
        case 4: return Cfg4::TH;
        case 5: return Cfg5::TH;
        case 6: return Cfg6::TH;
        case 7: return Cfg7::TH;
        case 8: return Cfg8::TH;
        case 9: return Cfg9::TH;
        case 10: return Cfg10::TH;
        case 11: return Cfg11::TH;
        case 12: return Cfg12::TH;
        case 13: return Cfg13::TH;
        case 14: return Cfg14::TH;
        case 15: return Cfg15::TH;
        case 16: return Cfg16::TH;
        case 17: return Cfg17::TH;
        default: return Cfg18::TH;
    }
}

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                 const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                 const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                 CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encoder() {
    static EncodeTiled fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
    }
    return fn;
}

}  // namespace

bool step_tiled_eligible(int H, int W, int K, int r_xy, int r_th, int storage) {
    const int align = storage == LOC_F32 ? 4 : 8;
    return r_xy == R && r_th == RT && K >= 8 && K <= LOC_MAX_K && W % align == 0 && W >= 8 && H >= 1;
}

int step_tiled_num_cfgs() { return 18; }

bool step_tiled_fuses_argmax(int cfg) { return cfg == 6 || cfg == 7 || (cfg >= 13 && cfg <= 16); }

int step_tiled_default_cfg(int H, int W, int K, int storage) {
    (void)K;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0)
        nsm = 152;
    // measured on GB300 (office plans): with many tiles per SM the 128-thread synchronous
    // configuration (3) is fastest for 16-bit storage, and its software-pipelined form (17, three
    // CTAs per SM) for FP32 (2048 x 2048 x 72: 0.79 against 0.83 ms; BF16 0.81 against 0.73)
    const long long cols = (W + TW - 1) / TW;
    if (cols * ((H + 15) / 16) >= 8LL * nsm) return storage == LOC_F32 ? 17 : 3;
    // with few tiles the warp-specialised pipelines, whose time follows the S/X rows (tile rows
    // + 4) that the busiest SM computes: 16-row tiles two per SM (6), 14-row tiles two per SM
    // with split producers (15), 28-row tiles one per SM (16); ties keep the earlier one
    const int cand[3][2] = {{6, Cfg6::TH}, {15, Cfg15::TH}, {16, Cfg16::TH}};
    int best = 6;
    long long best_cost = -1;
    for (const auto& c : cand) {
        const long long tiles = cols * ((H + c[1] - 1) / c[1]);
        const long long cost = (tiles + nsm - 1) / nsm * (c[1] + 2 * R);
        if (best_cost < 0 || cost < best_cost) {
            best = c[0];
            best_cost = cost;
        }
    }
    return best;
}

cudaError_t make_step_tmap(void* tmap_out, const void* B, int storage, int H, int W, int K, int cfg) {
    if (cfg < 1 || cfg > step_tiled_num_cfgs()) return cudaErrorInvalidValue;
    const bool paired = cfg >= 8 && cfg <= 12;    // the paired-column passes use a wider box
    const int bw = !paired ? BW : (storage == LOC_F32 ? pairs::pbw<float>() : pairs::pbw<__half>());
    return make_box_tmap(tmap_out, B, storage, H, W, K, bw, cfg_tile_rows(cfg) + 2 * R + 1);
}

cudaError_t make_box_tmap(void* tmap_out, const void* B, int storage, int H, int W, int K, int box_w, int box_h) {
    EncodeTiled enc = encoder();
    if (!enc) return cudaErrorNotSupported;
    const size_t e = storage == LOC_F32 ? 4 : 2;
    const CUtensorMapDataType dt = storage == LOC_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : storage == LOC_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                         : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    const cuuint64_t dims[3] = {(cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)K};
    const cuuint64_t strides[2] = {(cuuint64_t)W * e, (cuuint64_t)W * H * e};
    const cuuint32_t box[3] = {(cuuint32_t)box_w, (cuuint32_t)box_h, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(static_cast<CUtensorMap*>(tmap_out), dt, 3, const_cast<void*>(B), dims, strides, box,
                     estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

size_t step_tmap_bytes() { return sizeof(CUtensorMap); }

cudaError_t launch_step_tiled(const StepArgs& g, const void* tmap, int storage, int cfg, cudaStream_t st) {
    FastArgs a;
    memcpy(&a.tmap, tmap, sizeof(CUtensorMap));
    a.B_out = g.B_out;
    a.am_pv = g.am_pv;
    a.am_pi = g.am_pi;
    a.am_idx = g.am_idx;
    a.am_val = g.am_val;
    a.trav = g.trav;
    a.corr = g.corr;
    a.sd = g.sd;
    a.partials = g.partials;
    a.inv_uniform = g.inv_uniform;
    a.out_mult = g.out_mult;
    a.log_out_mult = g.log_out_mult;
    a.H = g.H;
    a.W = g.W;
    a.K = g.K;
    a.g0 = g.gx[R];
    a.g1 = g.gx[R + 1];
    a.g2 = g.gx[R + 2];
    for (int d = 0; d < RING; ++d) a.gt[d] = g.gt[d];
    for (int k = 0; k < g.K; ++k) a.sh[k] = g.sh[k];
    cudaError_t e;
    switch (storage) {
        case LOC_F32: e = launch_cfg<float>(cfg, a, g.W, g.H, st); break;
        case LOC_BF16: e = launch_cfg<__nv_bfloat16>(cfg, a, g.W, g.H, st); break;
        case LOC_F16: e = launch_cfg<__half>(cfg, a, g.W, g.H, st); break;
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace loc
