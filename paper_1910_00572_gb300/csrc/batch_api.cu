// C-ABI of the batched launch: many sessions of uneven H x W x K propagated by one persistent
// kernel per tick (batch.cu), the tick captured in CUDA graphs, the tile configuration picked
// by an autotuner that times the candidates on the batch itself.
//
// Per-session data that never changes (tensor maps of both ping-pong buffers, pointers, taps)
// is uploaded once.  Every tick the host runs each session's odometry bookkeeping (Section
// III-A, the same code as loc_step), writes the per-tick headers, the list of sessions to
// propagate with the index of each one's first tile, and the Eq. 2-3 shift tables into one of
// two pinned buffers, and launches a graph whose nodes copy that buffer to the device, reset
// the work-queue head and run the kernel.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "batch_core.h"

#define LOC_API extern "C" __attribute__((visibility("default")))

using namespace loc;

struct loc_batch_s {
    BatchCore core;
    bool failed = false;
    std::string err;
};

namespace loc {
namespace {

// Upload the per-session constants for configuration cfg.
cudaError_t build_static(BatchCore* c, int cfg) {
    const size_t n = c->sess.size();
    std::vector<BatchStatic> hs(n);
    int sh_off = 0;
    const int th = batch_tile_rows(cfg);
    c->tiles_all = 0;
    for (size_t s = 0; s < n; ++s) {
        const loc_session* h = c->sess[s];
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
        c->ntiles[s] = S.ntiles;
        c->tiles_all += S.ntiles;
    }
    if (c->tiles_all > (1LL << 30)) return cudaErrorInvalidValue;
    BatchCtl ctl{0, 0};
    cudaError_t e = cudaMemcpyAsync(c->d_static, hs.data(), sizeof(BatchStatic) * n, cudaMemcpyHostToDevice, c->bs);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_ctl, &ctl, sizeof(ctl), cudaMemcpyHostToDevice, c->bs);
    if (e == cudaSuccess) e = batch_prepare(c->storage, cfg, &c->grid);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->bs);
    if (e == cudaSuccess) c->cfg = cfg;
    return e;
}

// The work list of a tick: active sessions in work order (decreasing K, so the longest tiles
// are taken first; a session's tiles are consecutive, so tiles sharing halo rows run close
// together and the rows stay in L2).
void fill_list(BatchCore* c, void* buf, const std::vector<char>& active) {
    unsigned char* b = static_cast<unsigned char*>(buf);
    BatchList* list = reinterpret_cast<BatchList*>(b + c->lay.list_off);
    BatchActive* act = reinterpret_cast<BatchActive*>(b + c->lay.act_off);
    int na = 0, start = 0;
    for (int s : c->order)
        if (active[s]) {
            act[na++] = BatchActive{s, start};
            start += c->ntiles[s];
        }
    list->n_active = na;
    list->total = start;
}

// The tick's device work: copy the pinned buffer, reset the queue head, run the kernel.
cudaError_t enqueue_tick(BatchCore* c, int which, int dry) {
    cudaError_t e = cudaMemcpyAsync(c->d_tick, c->h_tick[which], c->lay.bytes, cudaMemcpyHostToDevice, c->bs);
    if (e == cudaSuccess) e = cudaMemsetAsync(&c->d_ctl->head, 0, sizeof(int), c->bs);
    if (e == cudaSuccess) e = launch_batch(c->storage, c->cfg, c->grid, c->d_static, c->d_tick, c->lay, c->d_ctl, dry, c->bs);
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

std::vector<long long> tune_key(const BatchCore* c) {
    std::vector<long long> shapes;
    for (const loc_session* h : c->sess)
        shapes.push_back(((long long)h->p.H << 40) | ((long long)h->p.W << 16) | h->p.K);
    std::sort(shapes.begin(), shapes.end());
    shapes.insert(shapes.begin(), (long long)c->storage);
    return shapes;
}

cudaError_t autotune(BatchCore* c) {
    const std::vector<long long> key = tune_key(c);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto hit = g_tuned.find(key);
        if (hit != g_tuned.end()) {
            std::memcpy(c->tune_ms, hit->second.ms, sizeof(c->tune_ms));
            return build_static(c, hit->second.cfg);
        }
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best = 1e30f;
    int best_cfg = 0;
    const std::vector<char> all(c->sess.size(), 1);
    BatchTick* ht = static_cast<BatchTick*>(c->h_tick[0]);
    for (size_t s = 0; s < c->sess.size(); ++s) ht[s] = BatchTick{c->sess[s]->cur, 0, 0, 0};
    std::memset(static_cast<unsigned char*>(c->h_tick[0]) + c->lay.shifts_off, 0, c->lay.bytes - c->lay.shifts_off);
    for (int cfg = 1; cfg <= batch_num_cfgs() && e == cudaSuccess; ++cfg) {
        e = build_static(c, cfg);
        if (e != cudaSuccess) break;
        fill_list(c, c->h_tick[0], all);
        e = enqueue_tick(c, 0, 1);
        if (e == cudaSuccess) e = cudaEventRecord(e0, c->bs);
        for (int r = 0; r < 3 && e == cudaSuccess; ++r) e = enqueue_tick(c, 0, 1);
        if (e == cudaSuccess) e = cudaEventRecord(e1, c->bs);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) break;
        c->tune_ms[cfg - 1] = ms / 3.0f;
        if (ms < best) {
            best = ms;
            best_cfg = cfg;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return e;
    BatchCtl ctl{};
    e = cudaMemcpy(&ctl, c->d_ctl, sizeof(ctl), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return e;
    if (ctl.status) return cudaErrorLaunchTimeout;   // a bounded wait gave up during tuning
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        Tuned t{best_cfg, {}};
        std::memcpy(t.ms, c->tune_ms, sizeof(t.ms));
        g_tuned[key] = t;
    }
    return build_static(c, best_cfg);
}

cudaError_t capture(BatchCore* c) {
    for (int w = 0; w < 2; ++w) {
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(c->bs, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return e;
        const cudaError_t e2 = enqueue_tick(c, w, 0);
        e = cudaStreamEndCapture(c->bs, &g);
        if (e2 != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return e2;
        }
        if (e != cudaSuccess) return e;
        e = cudaGraphInstantiate(&c->graph[w], g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

std::string batch_check(loc_session* const* sessions, int n) {
    if (!sessions || n <= 0) return "no sessions";
    int dev = 0;
    cudaGetDevice(&dev);
    for (int s = 0; s < n; ++s) {
        loc_session* h = sessions[s];
        if (!h) return "a session is null";
        if (h->failed) return "a session failed earlier: " + h->err;
        if (!step_tiled_eligible(h->p.H, h->p.W, h->p.K, h->r_xy, h->r_th, h->p.storage) ||
            h->p.kernel == LOC_KERNEL_GENERIC || h->aniso)
            return "batched sessions need the tiled kernel (radii 2/3, K >= 8, aligned W)";
        if (h->p.storage != sessions[0]->p.storage || h->stream != sessions[0]->stream || h->device != dev)
            return "sessions of a batch share one storage type, stream and device";
        for (int q = 0; q < s; ++q)
            if (sessions[q] == h) return "a session appears twice";
    }
    return "";
}

cudaError_t batch_init(BatchCore* c, loc_session* const* sessions, int n, int tile, bool use_graph) {
    int sum_k = 0;
    for (int s = 0; s < n; ++s) {
        c->sess.push_back(sessions[s]);
        c->sh_off.push_back(sum_k);
        sum_k += sessions[s]->p.K;
        c->order.push_back(s);
    }
    std::stable_sort(c->order.begin(), c->order.end(),
                     [&](int a, int b) { return c->sess[a]->p.K > c->sess[b]->p.K; });
    c->ntiles.assign((size_t)n, 0);
    c->storage = sessions[0]->p.storage;
    c->user = sessions[0]->stream;
    c->lay = batch_tick_layout(n, sum_k);
    // a stream of the batch's own (blocking, so ordered with the legacy default stream too)
    cudaError_t e = cudaStreamCreate(&c->bs);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_static, sizeof(BatchStatic) * (size_t)n);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_tick, c->lay.bytes);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_ctl, sizeof(BatchCtl));
    for (int w = 0; w < 2 && e == cudaSuccess; ++w) {
        e = cudaMallocHost(&c->h_tick[w], c->lay.bytes);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->done[w], cudaEventDisableTiming);
        if (e == cudaSuccess) std::memset(c->h_tick[w], 0, c->lay.bytes);
    }
    // the sessions' earlier work (creation, belief uploads) comes first
    if (e == cudaSuccess) e = cudaEventRecord(c->ev_in, c->user);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->bs, c->ev_in, 0);
    if (e == cudaSuccess) e = tile > 0 ? build_static(c, tile) : autotune(c);
    if (e == cudaSuccess && use_graph) {
        c->use_graph = true;
        e = capture(c);
    }
    return e;
}

void batch_release(BatchCore* c) {
    if (c->bs) cudaStreamSynchronize(c->bs);
    for (int w = 0; w < 2; ++w) {
        if (c->graph[w]) cudaGraphExecDestroy(c->graph[w]);
        if (c->h_tick[w]) cudaFreeHost(c->h_tick[w]);
        if (c->done[w]) cudaEventDestroy(c->done[w]);
        c->graph[w] = nullptr;
        c->h_tick[w] = nullptr;
        c->done[w] = nullptr;
    }
    if (c->d_static) cudaFree(c->d_static);
    if (c->d_tick) cudaFree(c->d_tick);
    if (c->d_ctl) cudaFree(c->d_ctl);
    if (c->ev_in) cudaEventDestroy(c->ev_in);
    if (c->ev_out) cudaEventDestroy(c->ev_out);
    if (c->bs) cudaStreamDestroy(c->bs);
    c->d_static = nullptr;
    c->d_tick = nullptr;
    c->d_ctl = nullptr;
    c->ev_in = c->ev_out = nullptr;
    c->bs = nullptr;
}

cudaError_t batch_begin(BatchCore* c, BatchTick** hdr, Shift** shifts) {
    const cudaError_t e = cudaEventSynchronize(c->done[c->parity]);
    unsigned char* b = static_cast<unsigned char*>(c->h_tick[c->parity]);
    *hdr = reinterpret_cast<BatchTick*>(b);
    *shifts = reinterpret_cast<Shift*>(b + c->lay.shifts_off);
    return e;
}

Shift* batch_shift_slot(BatchCore* c, Shift* shifts, int s) { return shifts + c->sh_off[s]; }

cudaError_t batch_launch(BatchCore* c, const std::vector<char>& active, cudaEvent_t done, bool join_user) {
    const int which = c->parity;
    fill_list(c, c->h_tick[which], active);
    const BatchList* list =
        reinterpret_cast<const BatchList*>(static_cast<unsigned char*>(c->h_tick[which]) + c->lay.list_off);
    if (list->n_active == 0) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    if (join_user) e = cudaEventRecord(c->ev_in, c->user);
    if (e == cudaSuccess && join_user) e = cudaStreamWaitEvent(c->bs, c->ev_in, 0);
    if (e == cudaSuccess) e = c->use_graph ? cudaGraphLaunch(c->graph[which], c->bs) : enqueue_tick(c, which, 0);
    if (e == cudaSuccess) e = cudaEventRecord(c->done[which], c->bs);
    if (e == cudaSuccess && done) e = cudaEventRecord(done, c->bs);
    if (e == cudaSuccess && join_user) e = cudaEventRecord(c->ev_out, c->bs);
    if (e == cudaSuccess && join_user) e = cudaStreamWaitEvent(c->user, c->ev_out, 0);
    if (e == cudaSuccess) {
        c->parity ^= 1;
        c->n_ticks += 1;
    }
    return e;
}

}  // namespace loc

namespace {

loc_status bfail(loc_batch b, loc_status code, const std::string& m) {
    if (b) {
        b->err = m;
        if (code == LOC_ERR_CUDA || code == LOC_ERR_TIMEOUT) b->failed = true;
    }
    set_thread_error(m.c_str());
    return code;
}

}  // namespace

LOC_API loc_status loc_batch_create(const loc_handle* sessions, int n, int tile, int use_graph, loc_batch* out) {
    if (!out) return bfail(nullptr, LOC_ERR_INVALID_ARG, "out is null");
    *out = nullptr;
    if (tile < 0 || tile > batch_num_cfgs()) return bfail(nullptr, LOC_ERR_INVALID_ARG, "tile configuration out of range");
    const std::string why = batch_check(sessions, n);
    if (!why.empty())
        return bfail(nullptr, why.rfind("a session failed", 0) == 0 ? LOC_ERR_STATE : LOC_ERR_INVALID_ARG, why);
    loc_batch b = new (std::nothrow) loc_batch_s();
    if (!b) return bfail(nullptr, LOC_ERR_OOM, "host allocation failed");
    const cudaError_t e = batch_init(&b->core, sessions, n, tile, use_graph != 0);
    if (e != cudaSuccess) {
        const std::string m = std::string("loc_batch_create: ") + cudaGetErrorString(e);
        cudaGetLastError();
        batch_release(&b->core);
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
    BatchCore* c = &b->core;
    const size_t n = c->sess.size();
    for (size_t s = 0; s < n; ++s) {
        if (!std::isfinite(u[s]) || !std::isfinite(v[s]) || !std::isfinite(w[s]))
            return bfail(b, LOC_ERR_INVALID_ARG, "odometry must be finite");
        if (c->sess[s]->failed) return bfail(b, LOC_ERR_STATE, "a session of the batch failed: " + c->sess[s]->err);
    }
    BatchTick* ht = nullptr;
    Shift* hs = nullptr;
    cudaError_t e = batch_begin(c, &ht, &hs);
    if (e != cudaSuccess) return bfail(b, LOC_ERR_CUDA, std::string("loc_batch_step: ") + cudaGetErrorString(e));
    std::vector<char> active(n, 0);
    int moved = 0;
    size_t off = 0;
    for (size_t s = 0; s < n; ++s) {
        loc_session* h = c->sess[s];
        if (odometry_advance(h, u[s], v[s], w[s])) {
            ht[s] = BatchTick{h->cur, 0, 0, 0};
            shift_table(h, hs + off);
            active[s] = 1;
            ++moved;
        }
        off += (size_t)h->p.K;
    }
    e = batch_launch(c, active, nullptr, true);
    if (e != cudaSuccess) {
        for (loc_session* h : c->sess) h->failed = true;
        return bfail(b, LOC_ERR_CUDA, std::string("loc_batch_step: ") + cudaGetErrorString(e));
    }
    for (size_t s = 0; s < n; ++s)
        if (active[s]) step_done(c->sess[s]);
    if (n_moved) *n_moved = moved;
    return moved ? LOC_OK : LOC_OK_DEFERRED;
}

LOC_API loc_status loc_batch_sync(loc_batch b) {
    if (!b) return bfail(nullptr, LOC_ERR_INVALID_ARG, "null batch");
    BatchCtl ctl{};
    cudaError_t e = cudaStreamSynchronize(b->core.bs);
    if (e == cudaSuccess) e = cudaMemcpy(&ctl, b->core.d_ctl, sizeof(ctl), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return bfail(b, LOC_ERR_CUDA, std::string("loc_batch_sync: ") + cudaGetErrorString(e));
    for (loc_session* h : b->core.sess) {
        const loc_status s = sync_and_check(h);
        if (s < 0) return bfail(b, s, "a session of the batch failed: " + h->err);
    }
    if (ctl.status & LOC_DEV_ERR_TIMEOUT) return bfail(b, LOC_ERR_TIMEOUT, "device wait timed out");
    return LOC_OK;
}

LOC_API loc_status loc_batch_info(loc_batch b, int* tile, int* n_items, int* grid, float* tune_ms) {
    if (!b) return bfail(nullptr, LOC_ERR_INVALID_ARG, "null batch");
    if (tile) *tile = b->core.cfg;
    if (n_items) *n_items = (int)b->core.tiles_all;
    if (grid) *grid = b->core.grid;
    if (tune_ms)
        for (int c = 0; c < LOC_BATCH_CONFIGS; ++c) tune_ms[c] = b->core.tune_ms[c];
    return LOC_OK;
}

LOC_API loc_status loc_batch_destroy(loc_batch b) {
    if (!b) return LOC_OK;
    batch_release(&b->core);
    delete b;
    return LOC_OK;
}

LOC_API const char* loc_batch_last_error(loc_batch b) { return b ? b->err.c_str() : ""; }
