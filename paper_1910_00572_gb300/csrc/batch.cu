// Batched propagation: many sessions of uneven H x W x K stepped by one persistent launch.
//
// The grid is sized to the GPU (resident CTAs per SM x SMs).  Each CTA repeatedly takes the
// next (session, tile) item from a device work queue and runs the synchronous tiled pass
// (Algorithm 1's propagation, run_tile) on that session's tile; the CTA that finishes a session's last
// tile combines the session's FP64 tile partials into its normaliser Z (Eq. 9) in the same
// fixed order as a single-session launch, so a session's result does not depend on which
// other sessions share the launch.
#include "kernels.h"
#include "tiled_common.cuh"

namespace loc {
namespace {

using namespace tiled;

template <typename T, typename C>
__global__ void __launch_bounds__(C::NT, C::MINB)
batch_kernel(const BatchStatic* __restrict__ ss, const BatchTick* __restrict__ tk, const BatchList* __restrict__ list,
             const BatchActive* __restrict__ act, const Shift* __restrict__ shifts, BatchCtl* ctl, int dry) {
    constexpr int NT = C::NT, NSTAGE = C::NSTAGE;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const uint32_t base = su32(smem_raw);
    Smem<T, C>& sm = *reinterpret_cast<Smem<T, C>*>(smem_raw + (((base + 127u) & ~127u) - base));
    __shared__ int s_sess, s_tile, s_last;
    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int s = 0; s < NSTAGE; ++s) bar_init(&sm.bar[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    const int total = list->total, n_active = list->n_active;
    unsigned int gp = 0;                   // planes this CTA has loaded through the mbarriers
    for (;;) {
        if (tid == 0) {
            const int q = atomicAdd(&ctl->head, 1);
            int sess = -1, tile = 0;
            if (q < total) {
                int lo = 0, hi = n_active - 1;           // last entry with start <= q
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (act[mid].start <= q) lo = mid;
                    else hi = mid - 1;
                }
                sess = act[lo].s;
                tile = q - act[lo].start;
            }
            s_sess = sess;
            s_tile = tile;
        }
        __syncthreads();
        const int sess = s_sess, tile = s_tile;
        if (sess < 0) break;
        const BatchTick t = tk[sess];
        const BatchStatic& S = ss[sess];
        const CUtensorMap* tmap = reinterpret_cast<const CUtensorMap*>(S.tmap[t.cur]);
        TileJob j;
        j.tmap = tmap;
        j.sh = shifts + S.sh_off;
        j.o.B_out = S.B[1 - t.cur];
        j.o.H = S.H;
        j.o.W = S.W;
        j.o.K = S.K;
        j.trav = S.trav;
        j.corr = S.corr;
        j.gt = S.gt;
        // a dry run times the steady state (TMA input) whatever the session's restart flag
        j.reinit = dry ? 0 : S.sd->reinit;
        // restart: the input is M / (K n_free); read M and fold 1 / (K n_free) into the scale
        j.in_scale = (j.reinit ? S.inv_uniform : S.sd->inv_Z) * S.out_mult;
        j.g0 = S.g0;
        j.g1 = S.g1;
        j.g2 = S.g2;
        j.ty0 = (tile / S.ntx) * C::TH;
        j.tx0 = (tile % S.ntx) * TW;
        if (tid == 0)   // the tensor map lives in global memory, written by a copy before the launch
            asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tmap) : "memory");
        KahanF2 acc;
        int p_stop = 0, next_issue = 0;
        if (!run_tile<T, C>(sm, j, gp, acc, p_stop, next_issue)) {
            // a TMA wait gave up: flag the launch and the session, let the copies in flight land
            // (bounded) and leave; the session's Z is not updated
            if (tid == 0) {
                atomicOr(&ctl->status, LOC_DEV_ERR_TIMEOUT);
                atomicOr(&S.sd->status, LOC_DEV_ERR_TIMEOUT);
                for (int q = p_stop; q < next_issue; ++q) {
                    const unsigned int g = gp + (unsigned int)q;
                    bar_wait(&sm.bar[g % NSTAGE], (g / NSTAGE) & 1u);
                }
            }
            __syncthreads();
            return;
        }
        if (!j.reinit) gp += (unsigned int)S.K;
        const double bt = block_sum<NT>(acc.value(), sm.red);
        if (dry) continue;                 // block_sum ended with a barrier
        if (tid == 0) {
            S.partials[tile] = bt;
            __threadfence();
            s_last = atomicAdd(&S.sd->counter, 1u) == (unsigned int)(S.ntiles - 1);
        }
        __syncthreads();
        if (s_last) {
            // the session's last tile: every partial is visible; sum them as finish_sum does
            __threadfence();
            double sum = 0.0;
            for (int b = tid; b < S.ntiles; b += NT) sum += ((volatile double*)S.partials)[b];
            const double Z = block_sum<NT>(sum, sm.red);
            if (tid == 0) {
                SessionDev* sd = S.sd;
                sd->counter = 0u;
                sd->n_prop += 1;
                if (Z > 0.0 && isfinite(Z)) {
                    sd->Z = Z;
                    sd->inv_Z = (float)(1.0 / Z);
                    sd->logscale += log(Z) - S.log_out_mult;
                    sd->reinit = 0;
                } else {
                    if (!isfinite(Z)) sd->status |= LOC_DEV_ERR_NONFINITE_Z;
                    sd->Z = 1.0;
                    sd->inv_Z = 1.0f;
                    sd->reinit = 1;
                    sd->n_reinit += 1;
                }
            }
        }
        __syncthreads();                   // s_last, s_sess and s_tile are rewritten next iteration
    }
}

// The candidates: the synchronous tile configurations 1-3 of the single-session kernel.
using BCfg1 = Cfg<32, 4, 3, 16, 3, 2>;
using BCfg2 = Cfg<16, 2, 2, 8, 3, 3>;
using BCfg3 = Cfg<16, 4, 4, 16, 3, 4>;

template <typename T, typename C>
cudaError_t prepare_typed(int* grid) {
    const size_t sb = sizeof(Smem<T, C>) + 128;
    cudaError_t e = cudaFuncSetAttribute(batch_kernel<T, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sb);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, occ = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, batch_kernel<T, C>, C::NT, sb);
    if (e != cudaSuccess) return e;
    *grid = (occ > 0 ? occ : 1) * sms;
    return cudaSuccess;
}

template <typename T, typename C>
cudaError_t launch_typed(int grid, const BatchStatic* ss, const void* tick, const BatchLayout& lay, BatchCtl* ctl,
                         int dry, cudaStream_t st) {
    const size_t sb = sizeof(Smem<T, C>) + 128;
    const unsigned char* b = static_cast<const unsigned char*>(tick);
    batch_kernel<T, C><<<grid, C::NT, sb, st>>>(ss, reinterpret_cast<const BatchTick*>(b),
                                                 reinterpret_cast<const BatchList*>(b + lay.list_off),
                                                 reinterpret_cast<const BatchActive*>(b + lay.act_off),
                                                 reinterpret_cast<const Shift*>(b + lay.shifts_off), ctl, dry);
    return cudaGetLastError();
}

template <typename T>
cudaError_t prepare_cfg(int cfg, int* grid) {
    switch (cfg) {
        case 1: return prepare_typed<T, BCfg1>(grid);
        case 2: return prepare_typed<T, BCfg2>(grid);
        case 3: return prepare_typed<T, BCfg3>(grid);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T>
cudaError_t launch_cfg(int cfg, int grid, const BatchStatic* ss, const void* tick, const BatchLayout& lay,
                       BatchCtl* ctl, int dry, cudaStream_t st) {
    switch (cfg) {
        case 1: return launch_typed<T, BCfg1>(grid, ss, tick, lay, ctl, dry, st);
        case 2: return launch_typed<T, BCfg2>(grid, ss, tick, lay, ctl, dry, st);
        case 3: return launch_typed<T, BCfg3>(grid, ss, tick, lay, ctl, dry, st);
        default: return cudaErrorInvalidValue;
    }
}

size_t up16(size_t x) { return (x + 15) & ~(size_t)15; }

}  // namespace

int batch_num_cfgs() { return 3; }

int batch_tile_rows(int cfg) { return cfg == 1 ? BCfg1::TH : cfg == 2 ? BCfg2::TH : BCfg3::TH; }

cudaError_t batch_prepare(int storage, int cfg, int* grid) {
    switch (storage) {
        case LOC_F32: return prepare_cfg<float>(cfg, grid);
        case LOC_BF16: return prepare_cfg<__nv_bfloat16>(cfg, grid);
        case LOC_F16: return prepare_cfg<__half>(cfg, grid);
        default: return cudaErrorInvalidValue;
    }
}

BatchLayout batch_tick_layout(int n_sessions, int sum_k) {
    BatchLayout l;
    l.list_off = up16(sizeof(BatchTick) * (size_t)n_sessions);
    l.act_off = up16(l.list_off + sizeof(BatchList));
    l.shifts_off = up16(l.act_off + sizeof(BatchActive) * (size_t)n_sessions);
    l.bytes = l.shifts_off + sizeof(Shift) * (size_t)sum_k;
    return l;
}

cudaError_t launch_batch(int storage, int cfg, int grid, const BatchStatic* ss, const void* tick,
                         const BatchLayout& lay, BatchCtl* ctl, int dry, cudaStream_t st) {
    if (grid <= 0) return cudaErrorInvalidValue;
    switch (storage) {
        case LOC_F32: return launch_cfg<float>(cfg, grid, ss, tick, lay, ctl, dry, st);
        case LOC_BF16: return launch_cfg<__nv_bfloat16>(cfg, grid, ss, tick, lay, ctl, dry, st);
        case LOC_F16: return launch_cfg<__half>(cfg, grid, ss, tick, lay, ctl, dry, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace loc
