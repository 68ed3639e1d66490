// C-ABI of the batched launch: many sessions of uneven H x W x K propagated by one persistent
// kernel per tick (batch.cu), the tick captured in CUDA graphs, the tile configuration picked
// by an autotuner that times the candidates on the batch itself.
//
// Per-session data that never changes (tensor maps of both ping-pong buffers, pointers, taps)
// is uploaded once.  Every tick the host runs each session's odometry bookkeeping (Section
// III-A, the same code as loc_step), writes the per-tick headers and the Eq. 2-3 shift tables
// into one of two pinned buffers, and launches a graph whose nodes copy that buffer to the
// device, reset the work-queue head and run the kernel.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "session.h"

#define LOC_API extern "C" __attribute__((visibility("default")))

using namespace loc;

struct loc_batch_s {
    std::vector<loc_session*> sess;
    int storage = LOC_F32;
    cudaStream_t user = nullptr;           // the sessions' stream
    cudaStream_t bs = nullptr;             // the batch's own stream (capturable)
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    int cfg = 0, grid = 0;
    float tune_ms[8] = {};
    size_t shifts_off = 0, tick_bytes = 0;
    BatchStatic* d_static = nullptr;
    void* d_tick = nullptr;
    void* h_tick[2] = {nullptr, nullptr};  // pinned, used by alternate ticks
    cudaEvent_t done[2] = {nullptr, nullptr};
    BatchItem* d_items = nullptr;
    int n_items = 0;
    BatchCtl* d_ctl = nullptr;
    bool use_graph = false;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int parity = 0;
    long long n_ticks = 0;
    bool failed = false;
    std::string err;
};

namespace {

loc_status bfail(loc_batch b, loc_status code, const std::string& m) {
    if (b) {
        b->err = m;
        if (code == LOC_ERR_CUDA || code == LOC_ERR_TIMEOUT) b->failed = true;
    }
    set_thread_error(m.c_str());
    return code;
}

BatchTick* ticks(void* buf) { return static_cast<BatchTick*>(buf); }
Shift* shifts(const loc_batch b, void* buf) {
    return reinterpret_cast<Shift*>(static_cast<unsigned char*>(buf) + b->shifts_off);
}

// Upload the per-session constants and the work list for configuration cfg.  Items are
// ordered by session, sessions by decreasing K (the per-tile cost), so the longest tiles are
// taken first and each session's tiles run close together (shared halo rows stay in L2).
cudaError_t build_static(loc_batch b, int cfg) {
    const size_t n = b->sess.size();
    std::vector<BatchStatic> hs(n);
    std::vector<int> order(n);
    int sh_off = 0;
    const int th = batch_tile_rows(cfg);
    for (size_t s = 0; s < n; ++s) {
        const loc_session* h = b->sess[s];
        BatchStatic& S = hs[s];
        std::memset(&S, 0, sizeof(S));
        for (int k = 0; k < 2; ++k) {
            cudaError_t e = make_step_tmap(S.tmap[k], h->B[k], h->p.storage, h->p.H, h->p.W, h->p.K, cfg);
            if (e != cudaSuccess) return e;
            S.B[k] = h->B[k];
        }
        S.trav = h->trav;
        S.corr = h->corr;
        S.sd = h->sd;
        S.partials = h->partials;
        S.inv_uniform = h->inv_uniform;
        S.out_mult = storage_mult(h->p.storage);
        S.log_out_mult = std::log((double)S.out_mult);
        S.H = h->p.H;
        S.W = h->p.W;
        S.K = h->p.K;
        S.ntx = (h->p.W + 63) / 64;
        S.ntiles = S.ntx * ((h->p.H + th - 1) / th);
        if ((unsigned int)S.ntiles > h->nparts) return cudaErrorInvalidValue;
        S.sh_off = sh_off;
        sh_off += h->p.K;
        S.g0 = h->gx[h->r_xy];
        S.g1 = h->gx[h->r_xy + 1];
        S.g2 = h->gx[h->r_xy + 2];
        for (int d = 0; d < 7; ++d) S.gt[d] = h->gt[d];
        order[s] = (int)s;
    }
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return hs[a].K > hs[c].K; });
    std::vector<BatchItem> items;
    for (int s : order)
        for (int t = 0; t < hs[s].ntiles; ++t) items.push_back(BatchItem{s, t});
    b->n_items = (int)items.size();
    BatchCtl ctl{0, b->n_items, 0, 0};
    cudaError_t e = cudaMemcpyAsync(b->d_static, hs.data(), sizeof(BatchStatic) * n, cudaMemcpyHostToDevice, b->bs);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_items, items.data(), sizeof(BatchItem) * items.size(), cudaMemcpyHostToDevice, b->bs);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_ctl, &ctl, sizeof(ctl), cudaMemcpyHostToDevice, b->bs);
    if (e == cudaSuccess) e = batch_prepare(b->storage, cfg, &b->grid);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->bs);
    if (e == cudaSuccess) b->cfg = cfg;
    return e;
}

// The tick's device work: copy the pinned buffer, reset the queue head, run the kernel.
cudaError_t enqueue_tick(loc_batch b, int which, int dry) {
    cudaError_t e = cudaMemcpyAsync(b->d_tick, b->h_tick[which], b->tick_bytes, cudaMemcpyHostToDevice, b->bs);
    if (e == cudaSuccess) e = cudaMemsetAsync(&b->d_ctl->head, 0, sizeof(int), b->bs);
    if (e == cudaSuccess)
        e = launch_batch(b->storage, b->cfg, b->grid, b->d_static, b->d_tick, b->shifts_off, b->d_items, b->d_ctl,
                         dry, b->bs);
    return e;
}

// Autotuner.  Every candidate configuration runs the whole batch in dry-run mode (every tile
// computed through the TMA path, outputs to the free ping-pong buffers, no session state
// changed): one warm-up launch, then the mean of three timed launches.  The fastest is kept
// and remembered for this storage type and multiset of (H, W, K).
struct Tuned {
    int cfg;
    float ms[8];
};
std::mutex g_tune_mu;
std::map<std::vector<long long>, Tuned> g_tuned;

std::vector<long long> tune_key(const loc_batch b) {
    std::vector<long long> shapes;
    for (const loc_session* h : b->sess)
        shapes.push_back(((long long)h->p.H << 40) | ((long long)h->p.W << 16) | h->p.K);
    std::sort(shapes.begin(), shapes.end());
    shapes.insert(shapes.begin(), (long long)b->storage);
    return shapes;
}

cudaError_t autotune(loc_batch b) {
    const std::vector<long long> key = tune_key(b);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto hit = g_tuned.find(key);
        if (hit != g_tuned.end()) {
            std::memcpy(b->tune_ms, hit->second.ms, sizeof(b->tune_ms));
            return build_static(b, hit->second.cfg);
        }
    }
    BatchTick* ht = ticks(b->h_tick[0]);
    Shift* hs = shifts(b, b->h_tick[0]);
    for (size_t s = 0; s < b->sess.size(); ++s) ht[s] = BatchTick{b->sess[s]->cur, 1, 0u, 0};
    std::memset(hs, 0, b->tick_bytes - b->shifts_off);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best = 1e30f;
    int best_cfg = 0;
    for (int cfg = 1; cfg <= batch_num_cfgs() && e == cudaSuccess; ++cfg) {
        e = build_static(b, cfg);
        if (e == cudaSuccess) e = enqueue_tick(b, 0, 1);
        if (e == cudaSuccess) e = cudaEventRecord(e0, b->bs);
        for (int r = 0; r < 3 && e == cudaSuccess; ++r) e = enqueue_tick(b, 0, 1);
        if (e == cudaSuccess) e = cudaEventRecord(e1, b->bs);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) break;
        b->tune_ms[cfg - 1] = ms / 3.0f;
        if (ms < best) {
            best = ms;
            best_cfg = cfg;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return e;
    int st = 0;
    e = cudaMemcpy(&st, &b->d_ctl->status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return e;
    if (st) return cudaErrorLaunchTimeout;           // a bounded wait gave up during tuning
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        Tuned t{best_cfg, {}};
        std::memcpy(t.ms, b->tune_ms, sizeof(t.ms));
        g_tuned[key] = t;
    }
    return build_static(b, best_cfg);
}

cudaError_t capture(loc_batch b) {
    for (int w = 0; w < 2; ++w) {
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(b->bs, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return e;
        const cudaError_t e2 = enqueue_tick(b, w, 0);
        e = cudaStreamEndCapture(b->bs, &g);
        if (e2 != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return e2;
        }
        if (e != cudaSuccess) return e;
        e = cudaGraphInstantiate(&b->graph[w], g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

void release(loc_batch b) {
    if (b->bs) cudaStreamSynchronize(b->bs);
    for (int w = 0; w < 2; ++w) {
        if (b->graph[w]) cudaGraphExecDestroy(b->graph[w]);
        if (b->h_tick[w]) cudaFreeHost(b->h_tick[w]);
        if (b->done[w]) cudaEventDestroy(b->done[w]);
    }
    if (b->d_static) cudaFree(b->d_static);
    if (b->d_tick) cudaFree(b->d_tick);
    if (b->d_items) cudaFree(b->d_items);
    if (b->d_ctl) cudaFree(b->d_ctl);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    if (b->bs) cudaStreamDestroy(b->bs);
}

}  // namespace

LOC_API loc_status loc_batch_create(const loc_handle* sessions, int n, int tile, int use_graph, loc_batch* out) {
    if (!out) return bfail(nullptr, LOC_ERR_INVALID_ARG, "out is null");
    *out = nullptr;
    if (!sessions || n <= 0) return bfail(nullptr, LOC_ERR_INVALID_ARG, "no sessions");
    if (tile < 0 || tile > batch_num_cfgs()) return bfail(nullptr, LOC_ERR_INVALID_ARG, "tile configuration out of range");
    int dev = 0;
    cudaGetDevice(&dev);
    for (int s = 0; s < n; ++s) {
        loc_session* h = sessions[s];
        if (!h) return bfail(nullptr, LOC_ERR_INVALID_ARG, "a session is null");
        if (h->failed) return bfail(nullptr, LOC_ERR_STATE, "a session failed earlier: " + h->err);
        if (!step_tiled_eligible(h->p.H, h->p.W, h->p.K, h->r_xy, h->r_th, h->p.storage) ||
            h->p.kernel == LOC_KERNEL_GENERIC)
            return bfail(nullptr, LOC_ERR_INVALID_ARG,
                         "batched sessions need the tiled kernel (radii 2/3, K >= 8, aligned W)");
        if (h->p.storage != sessions[0]->p.storage || h->stream != sessions[0]->stream || h->device != dev)
            return bfail(nullptr, LOC_ERR_INVALID_ARG, "sessions of a batch share one storage type, stream and device");
        for (int q = 0; q < s; ++q)
            if (sessions[q] == h) return bfail(nullptr, LOC_ERR_INVALID_ARG, "a session appears twice");
    }
    loc_batch b = new (std::nothrow) loc_batch_s();
    if (!b) return bfail(nullptr, LOC_ERR_OOM, "host allocation failed");
    size_t sum_k = 0, max_items = 0;
    for (int s = 0; s < n; ++s) {
        loc_session* h = sessions[s];
        b->sess.push_back(h);
        sum_k += (size_t)h->p.K;
        size_t most = 0;
        for (int c = 1; c <= batch_num_cfgs(); ++c) {
            const int th = batch_tile_rows(c);
            most = std::max(most, (size_t)((h->p.W + 63) / 64) * (size_t)((h->p.H + th - 1) / th));
        }
        max_items += most;
    }
    b->storage = sessions[0]->p.storage;
    b->user = sessions[0]->stream;
    b->shifts_off = (sizeof(BatchTick) * (size_t)n + 15) & ~(size_t)15;
    b->tick_bytes = b->shifts_off + sizeof(Shift) * sum_k;
    // a stream of the batch's own (blocking, so ordered with the legacy default stream too)
    cudaError_t e = cudaStreamCreate(&b->bs);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_static, sizeof(BatchStatic) * (size_t)n);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_tick, b->tick_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_items, sizeof(BatchItem) * max_items);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_ctl, sizeof(BatchCtl));
    for (int w = 0; w < 2 && e == cudaSuccess; ++w) {
        e = cudaMallocHost(&b->h_tick[w], b->tick_bytes);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->done[w], cudaEventDisableTiming);
        if (e == cudaSuccess) std::memset(b->h_tick[w], 0, b->tick_bytes);
    }
    // the sessions' earlier work (creation, belief uploads) comes first
    if (e == cudaSuccess) e = cudaEventRecord(b->ev_in, b->user);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->bs, b->ev_in, 0);
    if (e == cudaSuccess) e = tile > 0 ? build_static(b, tile) : autotune(b);
    if (e == cudaSuccess && use_graph) {
        b->use_graph = true;
        e = capture(b);
    }
    if (e != cudaSuccess) {
        const std::string m = std::string("loc_batch_create: ") + cudaGetErrorString(e);
        cudaGetLastError();
        release(b);
        delete b;
        return bfail(nullptr, e == cudaErrorMemoryAllocation ? LOC_ERR_OOM : LOC_ERR_CUDA, m);
    }
    *out = b;
    return LOC_OK;
}

LOC_API loc_status loc_batch_step(loc_batch b, const double* u, const double* v, const double* w, int* n_moved) {
    if (n_moved) *n_moved = 0;
    if (!b) return bfail(nullptr, LOC_ERR_INVALID_ARG, "null batch");
    if (b->failed) return bfail(b, LOC_ERR_STATE, "batch failed earlier: " + b->err);
    if (!u || !v || !w) return bfail(b, LOC_ERR_INVALID_ARG, "null odometry arrays");
    const size_t n = b->sess.size();
    for (size_t s = 0; s < n; ++s) {
        if (!std::isfinite(u[s]) || !std::isfinite(v[s]) || !std::isfinite(w[s]))
            return bfail(b, LOC_ERR_INVALID_ARG, "odometry must be finite");
        if (b->sess[s]->failed) return bfail(b, LOC_ERR_STATE, "a session of the batch failed: " + b->sess[s]->err);
    }
    const int which = b->parity;
    // the pinned buffer of this parity was read by the copy two ticks ago
    cudaError_t e = cudaEventSynchronize(b->done[which]);
    if (e != cudaSuccess) return bfail(b, LOC_ERR_CUDA, std::string("loc_batch_step: ") + cudaGetErrorString(e));
    BatchTick* ht = ticks(b->h_tick[which]);
    Shift* hs = shifts(b, b->h_tick[which]);
    int moved = 0;
    size_t off = 0;
    for (size_t s = 0; s < n; ++s) {
        loc_session* h = b->sess[s];
        const bool go = odometry_advance(h, u[s], v[s], w[s]);
        ht[s] = BatchTick{h->cur, go ? 1 : 0, step_seed(h), 0};
        if (go) {
            shift_table(h, hs + off);
            ++moved;
        }
        off += (size_t)h->p.K;
    }
    if (moved) {
        e = cudaEventRecord(b->ev_in, b->user);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->bs, b->ev_in, 0);
        if (e == cudaSuccess) e = b->use_graph ? cudaGraphLaunch(b->graph[which], b->bs) : enqueue_tick(b, which, 0);
        if (e == cudaSuccess) e = cudaEventRecord(b->done[which], b->bs);
        if (e == cudaSuccess) e = cudaEventRecord(b->ev_out, b->bs);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->user, b->ev_out, 0);
        if (e != cudaSuccess) {
            for (loc_session* h : b->sess) h->failed = true;
            return bfail(b, LOC_ERR_CUDA, std::string("loc_batch_step: ") + cudaGetErrorString(e));
        }
        for (size_t s = 0; s < n; ++s)
            if (ht[s].active) step_done(b->sess[s]);
        b->parity ^= 1;
        b->n_ticks += 1;
    }
    if (n_moved) *n_moved = moved;
    return moved ? LOC_OK : LOC_OK_DEFERRED;
}

LOC_API loc_status loc_batch_sync(loc_batch b) {
    if (!b) return bfail(nullptr, LOC_ERR_INVALID_ARG, "null batch");
    cudaError_t e = cudaStreamSynchronize(b->bs);
    int st = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&st, &b->d_ctl->status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return bfail(b, LOC_ERR_CUDA, std::string("loc_batch_sync: ") + cudaGetErrorString(e));
    for (loc_session* h : b->sess) {
        const loc_status s = sync_and_check(h);
        if (s != LOC_OK) return bfail(b, s, "a session of the batch failed: " + h->err);
    }
    if (st & LOC_DEV_ERR_TIMEOUT) return bfail(b, LOC_ERR_TIMEOUT, "device wait timed out");
    return LOC_OK;
}

LOC_API loc_status loc_batch_info(loc_batch b, int* tile, int* n_items, int* grid, float* tune_ms) {
    if (!b) return bfail(nullptr, LOC_ERR_INVALID_ARG, "null batch");
    if (tile) *tile = b->cfg;
    if (n_items) *n_items = b->n_items;
    if (grid) *grid = b->grid;
    if (tune_ms)
        for (int c = 0; c < LOC_BATCH_CONFIGS; ++c) tune_ms[c] = b->tune_ms[c];
    return LOC_OK;
}

LOC_API loc_status loc_batch_destroy(loc_batch b) {
    if (!b) return LOC_OK;
    release(b);
    delete b;
    return LOC_OK;
}

LOC_API const char* loc_batch_last_error(loc_batch b) { return b ? b->err.c_str() : ""; }
