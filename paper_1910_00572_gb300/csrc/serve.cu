// Serving loop: robot sessions stepped as their odometry and scan messages arrive.
//
// Threads.  Client threads submit messages into per-session queues (loc_server_odometry,
// loc_server_scan).  One worker thread owns every session's host state and every launch: each
// iteration it (1) closes sessions whose queues ran empty and admits pending sessions, first
// come first served, while their device bytes fit the budget (rebuilding the batched launch
// when the set changes), (2) takes work from each admitted session's queue -- odometry
// messages run through the session's Alg. 1 gate one by one until one opens it, with at most
// one scan message before that -- and (3) launches it: each scan update on the session's own
// stream, then all propagations of the tick in one persistent batched launch.
// A completion thread polls the events recorded after each piece of work and timestamps it.
//
// Ordering.  A session's work runs in message order: a batch waits for the scan updates
// of its sessions launched since their last batch (this tick's included), and a scan update
// waits for the batch that last propagated its session.  Because a session is propagated at most once per tick and its
// gate only sees its own messages, the propagation points, the rounding keys and therefore the
// results do not depend on the load or on the other sessions.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <functional>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "batch_core.h"

#define LOC_API extern "C" __attribute__((visibility("default")))

using namespace loc;

namespace {

enum { MSG_ODO = 0, MSG_SCAN = 1 };

struct SrvScan {
    std::vector<float> ranges;
    double angle_min = 0, angle_inc = 0, r_max = 0, sigma_r = 0;
    int stride = 1;
};

struct SrvMsg {
    int kind = MSG_ODO;
    double u = 0, v = 0, w = 0;
    double t_arr = 0;
    SrvScan* scan = nullptr;           // owned while queued
    double theta = 0;                  // scan taken into a tick: the session's heading then
};

struct SrvSession {
    int id = -1;
    int state = LOC_SESSION_PENDING;
    bool closing = false;
    std::vector<uint8_t> occ;          // kept until admission
    loc_params p{};
    size_t bytes = 0;
    loc_session* h = nullptr;
    std::deque<SrvMsg> q;
    int stream_idx = 0;
    int ci = -1;                       // index in the batched launch
    long long last_prop_tick = -1;
    cudaEvent_t scan_ev = nullptr;     // recorded after the session's latest scan update
    // The pool stream a session's scans and plain steps run on changes from tick to tick, so
    // that each tick's work spreads over every stream; tail_ev (recorded after the session's
    // latest work on a pool stream) orders the next stream after the previous one.
    cudaEvent_t tail_ev = nullptr;
    bool tail_valid = false;
    long long scan_tick = -1;          // tick of the session's latest scan
    bool scan_pending = false;         // a scan update was launched since its last propagation
};

// Categories of timed device work: the batched launch, a scan update, a plain loc_step.
enum { WORK_BATCH = 0, WORK_SCAN = 1, WORK_PLAIN = 2 };

struct Inflight {
    cudaEvent_t ev;
    int kind;
    std::vector<double> t_arr;
    cudaEvent_t ev0 = nullptr;         // timing start (recorded where the work could begin)
    int work = WORK_BATCH;
    double bytes = 0.0;                // algorithmic HBM bytes of the work (propagations)
};

constexpr int kRing = 64;              // batch events kept for scan ordering
constexpr size_t kScanThreads = 8;     // host threads preparing a tick's scan updates

double pct(std::vector<double> v, double q) {
    if (v.empty()) return 0.0;
    const size_t k = (size_t)std::min<double>((double)v.size() - 1, std::floor(q * (double)(v.size() - 1) + 0.5));
    std::nth_element(v.begin(), v.begin() + (long)k, v.end());
    return v[k];
}

}  // namespace

struct loc_server_s {
    loc_server_params prm{};
    int device = 0;
    std::chrono::steady_clock::time_point t0;
    // sessions and queues
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::vector<SrvSession*> sessions;
    std::deque<int> admit_q;
    size_t used_bytes = 0;
    bool stop = false;
    bool busy = false;                 // the worker holds work taken from the queues
    bool failed = false;
    std::string err;
    // worker-owned
    std::vector<cudaStream_t> pool;
    cudaEvent_t ring[kRing] = {};
    BatchCore core;
    bool core_live = false;
    int tuned_tile = 0;
    size_t tuned_at = 0;               // live sessions when the tile was last autotuned
    std::vector<SrvSession*> live;
    long long tick = 0;
    size_t scan_rr = 0, plain_rr = 0;  // next pool stream for a scan / a session's plain steps
    std::thread worker, completer;
    // helper threads for the scan phase of a tick, started once: the worker publishes a job
    // (generation gen), each helper runs it once, and the worker waits until pool_busy is 0
    std::vector<std::thread> pool_threads;
    std::mutex mu_pool;
    std::condition_variable cv_pool, cv_pool_done;
    std::function<void()> pool_job;
    long long pool_gen = 0;
    int pool_busy = 0;
    bool pool_stop = false;
    // completion tracking
    std::mutex mu_inf;
    std::deque<Inflight> inflight;
    std::vector<cudaEvent_t> ev_free;
    std::atomic<bool> stop_completer{false};
    // statistics (mu_st)
    std::mutex mu_st;
    std::vector<double> lat_step, lat_scan;
    long long n_ticks = 0, n_msgs = 0, n_props = 0, n_scans = 0, n_batched = 0, n_in_batches = 0;
    double cells = 0.0, first_s = -1.0, last_s = 0.0;
    // device time per category of work (event pairs) and the worker's host time per tick phase
    double dev_ms[3] = {0.0, 0.0, 0.0}, dev_bytes[3] = {0.0, 0.0, 0.0};
    long long dev_n[3] = {0, 0, 0};
    double host_gather_ms = 0.0, host_batch_ms = 0.0, host_scan_ms = 0.0, host_plain_ms = 0.0;

    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace {

loc_status sfail(loc_server s, loc_status code, const std::string& m) {
    if (s) {
        std::lock_guard<std::mutex> lk(s->mu);
        s->err = m;
    }
    set_thread_error(m.c_str());
    return code;
}

void set_failed(loc_server s, const std::string& m) {
    std::lock_guard<std::mutex> lk(s->mu);
    if (!s->failed) {
        s->failed = true;
        s->err = m;
    }
    s->cv_done.notify_all();
}

cudaEvent_t get_event(loc_server s) {
    {
        std::lock_guard<std::mutex> lk(s->mu_inf);
        if (!s->ev_free.empty()) {
            cudaEvent_t e = s->ev_free.back();
            s->ev_free.pop_back();
            return e;
        }
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;   // timing enabled: ends of timed work
    return e;
}

void push_inflight(loc_server s, cudaEvent_t ev, int kind, std::vector<double>&& t_arr, cudaEvent_t ev0 = nullptr,
                   int work = WORK_BATCH, double bytes = 0.0) {
    std::lock_guard<std::mutex> lk(s->mu_inf);
    Inflight f{ev, kind, std::move(t_arr)};
    f.ev0 = ev0;
    f.work = work;
    f.bytes = bytes;
    s->inflight.push_back(std::move(f));
}

double ms_since(std::chrono::steady_clock::time_point t) {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t).count();
}

void note_arrival(loc_server s, double t) {
    std::lock_guard<std::mutex> lk(s->mu_st);
    if (s->first_s < 0.0 || t < s->first_s) s->first_s = t;
}

// Completion thread: timestamps finished work as soon as its event has completed.
void completer_main(loc_server s) {
    cudaSetDevice(s->device);
    for (;;) {
        bool any = false, empty = false;
        std::string failure;
        {
            std::lock_guard<std::mutex> lk(s->mu_inf);
            for (auto it = s->inflight.begin(); it != s->inflight.end();) {
                const cudaError_t q = cudaEventQuery(it->ev);
                if (q == cudaErrorNotReady) {
                    ++it;
                    continue;
                }
                const double t = s->now();
                if (q != cudaSuccess) {
                    cudaGetLastError();
                    failure = std::string("device work failed: ") + cudaGetErrorString(q);
                }
                float dms = -1.0f;
                if (it->ev0 && q == cudaSuccess && cudaEventElapsedTime(&dms, it->ev0, it->ev) != cudaSuccess) {
                    cudaGetLastError();
                    dms = -1.0f;
                }
                {
                    std::lock_guard<std::mutex> ls(s->mu_st);
                    for (double a : it->t_arr) {
                        (it->kind == MSG_ODO ? s->lat_step : s->lat_scan).push_back((t - a) * 1e3);
                        s->n_msgs += 1;
                    }
                    s->last_s = std::max(s->last_s, t);
                    if (dms >= 0.0f) {
                        s->dev_ms[it->work] += dms;
                        s->dev_bytes[it->work] += it->bytes;
                        s->dev_n[it->work] += 1;
                    }
                }
                if (it->ev0) s->ev_free.push_back(it->ev0);
                s->ev_free.push_back(it->ev);
                it = s->inflight.erase(it);
                any = true;
            }
            empty = s->inflight.empty();
        }
        if (!failure.empty()) set_failed(s, failure);    // takes mu: never while holding mu_inf
        if (any) {
            std::lock_guard<std::mutex> lk(s->mu);
            s->cv_done.notify_all();
        }
        if (empty && s->stop_completer.load()) return;
        if (!any) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

cudaError_t sync_all(loc_server s) {
    cudaError_t e = cudaSuccess;
    if (s->core_live && s->core.bs) e = cudaStreamSynchronize(s->core.bs);
    for (cudaStream_t st : s->pool)
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e;
}

// Scan-phase helper: runs each published job once.
void pool_main(loc_server s) {
    cudaSetDevice(s->device);
    long long seen = 0;
    for (;;) {
        std::function<void()> job;
        {
            std::unique_lock<std::mutex> lk(s->mu_pool);
            s->cv_pool.wait(lk, [&] { return s->pool_stop || s->pool_gen != seen; });
            if (s->pool_stop) return;
            seen = s->pool_gen;
            job = s->pool_job;
        }
        job();
        std::lock_guard<std::mutex> lk(s->mu_pool);
        if (--s->pool_busy == 0) s->cv_pool_done.notify_all();
    }
}

// Runs job on the calling thread and on every helper, and returns when all are done.
void pool_run(loc_server s, const std::function<void()>& job) {
    {
        std::lock_guard<std::mutex> lk(s->mu_pool);
        s->pool_job = job;
        s->pool_busy = (int)s->pool_threads.size();
        s->pool_gen += 1;
    }
    s->cv_pool.notify_all();
    job();
    std::unique_lock<std::mutex> lk(s->mu_pool);
    s->cv_pool_done.wait(lk, [&] { return s->pool_busy == 0; });
    s->pool_job = nullptr;
}

// Closes drained sessions, admits pending ones, rebuilds the batched launch.  Worker thread.
bool membership(loc_server s) {
    std::vector<SrvSession*> to_close, to_admit;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        size_t used = s->used_bytes;
        for (SrvSession* ss : s->live)
            if (ss->closing && ss->q.empty()) {
                to_close.push_back(ss);
                used -= ss->bytes;
            }
        while (!s->admit_q.empty()) {
            SrvSession* ss = s->sessions[(size_t)s->admit_q.front()];
            if (ss->closing) {                   // closed before admission
                ss->state = LOC_SESSION_CLOSED;
                for (SrvMsg& m : ss->q) delete m.scan;
                ss->q.clear();
                s->admit_q.pop_front();
                continue;
            }
            if ((double)(used + ss->bytes) > s->prm.hbm_budget_bytes) break;
            used += ss->bytes;
            to_admit.push_back(ss);
            s->admit_q.pop_front();
        }
        if (!to_close.empty() || !to_admit.empty()) s->busy = true;   // drain waits for the change
    }
    if (to_close.empty() && to_admit.empty()) return true;
    if (sync_all(s) != cudaSuccess) {
        set_failed(s, "stream synchronisation failed");
        return false;
    }
    for (SrvSession* ss : to_close) {
        loc_destroy(ss->h);
        std::lock_guard<std::mutex> lk(s->mu);
        ss->h = nullptr;
        ss->state = LOC_SESSION_CLOSED;
        s->used_bytes -= ss->bytes;
    }
    for (SrvSession* ss : to_admit) {
        loc_params p = ss->p;
        p.stream = (void*)s->pool[(size_t)ss->stream_idx];
        loc_handle h = nullptr;
        const loc_status st = loc_create(ss->occ.data(), &p, &h);
        std::lock_guard<std::mutex> lk(s->mu);
        std::vector<uint8_t>().swap(ss->occ);
        if (st != LOC_OK) {
            ss->state = LOC_SESSION_FAILED;
            for (SrvMsg& m : ss->q) delete m.scan;
            ss->q.clear();
            continue;
        }
        bool ev_ok = true;
        for (cudaEvent_t* pe : {&ss->scan_ev, &ss->tail_ev})
            if (!*pe && cudaEventCreateWithFlags(pe, cudaEventDisableTiming) != cudaSuccess) {
                *pe = nullptr;
                ev_ok = false;
            }
        // the session's set-up ran on its first stream: later streams wait for it
        if (ev_ok) ev_ok = cudaEventRecord(ss->tail_ev, s->pool[(size_t)ss->stream_idx]) == cudaSuccess;
        if (!ev_ok) {
            loc_destroy(h);
            ss->state = LOC_SESSION_FAILED;
            for (SrvMsg& m : ss->q) delete m.scan;
            ss->q.clear();
            continue;
        }
        ss->h = h;
        ss->tail_valid = true;
        ss->state = LOC_SESSION_ACTIVE;
        s->used_bytes += ss->bytes;
    }
    std::vector<SrvSession*> live;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (SrvSession* ss : s->sessions)
            if (ss->state == LOC_SESSION_ACTIVE) live.push_back(ss);
    }
    if (s->prm.batching) {
        if (s->core_live) {
            batch_release(&s->core);
            s->core = BatchCore();
            s->core_live = false;
        }
        if (!live.empty()) {
            std::vector<loc_session*> hs;
            for (size_t i = 0; i < live.size(); ++i) {
                hs.push_back(live[i]->h);
                live[i]->ci = (int)i;
            }
            // autotune (prm.tile == 0) on the first batch and again whenever the number of
            // sessions has doubled since; otherwise keep the tuned configuration
            int tile = s->prm.tile;
            if (tile == 0 && s->tuned_tile > 0 && live.size() < 2 * s->tuned_at) tile = s->tuned_tile;
            if (tile == 0) s->tuned_at = live.size();
            const cudaError_t e = batch_init(&s->core, hs.data(), (int)hs.size(), tile, s->prm.use_graph != 0);
            s->core_live = true;
            if (e != cudaSuccess) {
                set_failed(s, std::string("batched launch setup: ") + cudaGetErrorString(e));
                return false;
            }
            s->tuned_tile = s->core.cfg;
            // the batch's stream starts after everything the sessions did so far
            if (sync_all(s) != cudaSuccess) {
                set_failed(s, "stream synchronisation failed");
                return false;
            }
        }
    }
    std::lock_guard<std::mutex> lk(s->mu);
    s->live = live;
    s->busy = false;
    s->cv_done.notify_all();
    return true;
}

struct TickWork {
    std::vector<std::pair<SrvSession*, double>> props;           // batched: gate opened
    std::vector<std::pair<SrvSession*, SrvMsg>> scans;
    std::vector<std::pair<SrvSession*, SrvMsg>> plain;           // plain path: odometry messages
    long long absorbed = 0;                                      // odometry kept back by the gate
    bool empty() const { return props.empty() && scans.empty() && plain.empty() && absorbed == 0; }
};

// Takes this tick's work from the queues (under the lock).  Worker thread.  Per session, in
// message order: odometry the gate absorbs, at most one scan, then odometry up to the first
// propagation.  A scan that follows the tick's propagation waits for the next tick, so the
// tick's scans can run before its propagations (launch).
void gather(loc_server s, TickWork& t) {
    for (SrvSession* ss : s->live) {
        bool prop = false, scanned = false;
        while (!ss->q.empty()) {
            SrvMsg& m = ss->q.front();
            if (m.kind == MSG_SCAN) {
                if (prop || scanned) break;
                // the tick's later odometry reaches the gate (and the heading) before the scan
                // is launched: the scan keeps the heading its own position in the stream gives
                if (ss->h) m.theta = ss->h->theta;
                t.scans.emplace_back(ss, m);
                ss->q.pop_front();
                scanned = true;
                continue;
            }
            if (!s->prm.batching) {                  // loc_step applies the gate itself
                t.plain.emplace_back(ss, m);
                ss->q.pop_front();
                prop = true;
                continue;
            }
            if (prop) break;
            const bool go = odometry_advance(ss->h, m.u, m.v, m.w);
            const double ta = m.t_arr;
            ss->q.pop_front();
            if (go) {
                t.props.emplace_back(ss, ta);
                prop = true;
            } else {
                t.absorbed += 1;
            }
        }
    }
}

// Moves a session's pool-stream work to stream k, after its work on the previous stream.
cudaError_t bind_stream(loc_server s, SrvSession* ss, int k) {
    if (ss->stream_idx == k) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    if (ss->tail_valid) e = cudaStreamWaitEvent(s->pool[(size_t)k], ss->tail_ev, 0);
    ss->stream_idx = k;
    ss->h->stream = s->pool[(size_t)k];
    return e;
}

// The tick's scan updates: distinct sessions, spread over the pool streams in turn, each after
// the batch that last propagated its session.  Their host work (direction tables, uploads,
// launches) runs on up to kScanThreads threads.
bool launch_scans(loc_server s, TickWork& t) {
    std::atomic<int> next{0};
    std::atomic<bool> bad{false};
    auto scan_worker = [&]() {
        cudaSetDevice(s->device);
        for (;;) {
            const int i = next.fetch_add(1);
            if (i >= (int)t.scans.size() || bad.load()) return;
            SrvSession* ss = t.scans[(size_t)i].first;
            SrvScan* sc = t.scans[(size_t)i].second.scan;
            // the tick's scans take the streams in turn
            cudaError_t we = bind_stream(s, ss, (int)((s->scan_rr + (size_t)i) % s->pool.size()));
            cudaStream_t ps = s->pool[(size_t)ss->stream_idx];
            ss->scan_tick = s->tick;
            if (we == cudaSuccess && s->prm.batching && ss->last_prop_tick >= 0)
                we = cudaStreamWaitEvent(ps, s->ring[ss->last_prop_tick % kRing], 0);
            cudaEvent_t ev0 = we == cudaSuccess ? get_event(s) : nullptr;
            if (we == cudaSuccess) we = ev0 ? cudaEventRecord(ev0, ps) : cudaErrorMemoryAllocation;
            if (we != cudaSuccess) {
                set_failed(s, std::string("scan ordering: ") + cudaGetErrorString(we));
                bad = true;
                return;
            }
            // the heading when the scan arrived; the session belongs to this helper until the
            // scan phase ends, and no other work of the tick reads its heading before then
            const double theta_now = ss->h->theta;
            ss->h->theta = t.scans[(size_t)i].second.theta;
            const loc_status st = loc_lidar_update(ss->h, sc->ranges.data(), (int)sc->ranges.size(), sc->angle_min,
                                                   sc->angle_inc, sc->r_max, sc->stride, sc->sigma_r);
            ss->h->theta = theta_now;
            delete sc;
            t.scans[(size_t)i].second.scan = nullptr;
            if (st < 0) {
                set_failed(s, std::string("loc_lidar_update: ") + loc_last_error(ss->h));
                bad = true;
                return;
            }
            cudaEvent_t ev = get_event(s);
            if (!ev || cudaEventRecord(ev, ps) != cudaSuccess || cudaEventRecord(ss->tail_ev, ps) != cudaSuccess ||
                (s->prm.batching && cudaEventRecord(ss->scan_ev, ps) != cudaSuccess)) {
                set_failed(s, "event record failed");
                bad = true;
                return;
            }
            ss->scan_pending = true;
            ss->tail_valid = true;
            {
                std::lock_guard<std::mutex> ls(s->mu_st);
                s->n_scans += 1;
            }
            push_inflight(s, ev, MSG_SCAN, std::vector<double>{t.scans[(size_t)i].second.t_arr}, ev0, WORK_SCAN);
        }
    };
    if (!t.scans.empty()) {
        const auto ts = std::chrono::steady_clock::now();
        // the largest maps first, on distinct streams: their dithering chains are the longest
        std::stable_sort(t.scans.begin(), t.scans.end(), [](const auto& a, const auto& b) {
            return (size_t)a.first->p.H * a.first->p.W > (size_t)b.first->p.H * b.first->p.W;
        });
        if (t.scans.size() == 1 || s->pool_threads.empty()) scan_worker();
        else pool_run(s, scan_worker);
        for (auto& pm : t.scans) delete pm.second.scan;     // left over after a failure
        if (bad.load()) return false;
        s->scan_rr += t.scans.size();
        std::lock_guard<std::mutex> ls(s->mu_st);
        s->host_scan_ms += ms_since(ts);
    }
    return true;
}

// The tick's propagations in one batched launch, after the scan updates of their sessions.
bool launch_batch(loc_server s, TickWork& t) {
    cudaError_t e = cudaSuccess;
    if (!t.props.empty()) {
        // the batch follows the scan updates of its sessions launched since their last batch
        for (auto& pr : t.props)
            if (pr.first->scan_pending && e == cudaSuccess) {
                e = cudaStreamWaitEvent(s->core.bs, pr.first->scan_ev, 0);
                pr.first->scan_pending = false;
            }
        const auto tb = std::chrono::steady_clock::now();
        BatchTick* ht = nullptr;
        Shift* hs = nullptr;
        if (e == cudaSuccess) e = batch_begin(&s->core, &ht, &hs);
        std::vector<char> active(s->core.sess.size(), 0);
        std::vector<double> arr;
        double cells = 0.0, bytes = 0.0;
        if (e == cudaSuccess) {
            for (auto& pr : t.props) {
                loc_session* h = pr.first->h;
                const int ci = pr.first->ci;
                ht[ci] = BatchTick{h->cur, 0, 0, 0};
                shift_table(h, batch_shift_slot(&s->core, hs, ci));
                active[(size_t)ci] = 1;
                arr.push_back(pr.second);
                const double hw = (double)h->p.H * h->p.W;
                cells += hw * h->p.K;
                bytes += hw * h->p.K * 2.0 * (double)h->elem + hw * 5.0;   // read + write X, map fields
            }
        }
        cudaEvent_t ev0 = e == cudaSuccess ? get_event(s) : nullptr;
        cudaEvent_t ev = e == cudaSuccess ? get_event(s) : nullptr;
        if (e == cudaSuccess && (!ev || !ev0)) e = cudaErrorMemoryAllocation;
        if (e == cudaSuccess) e = cudaEventRecord(ev0, s->core.bs);
        if (e == cudaSuccess) e = batch_launch(&s->core, active, ev, false);
        if (e == cudaSuccess) e = cudaEventRecord(s->ring[s->tick % kRing], s->core.bs);
        if (e != cudaSuccess) {
            set_failed(s, std::string("batched launch: ") + cudaGetErrorString(e));
            return false;
        }
        for (auto& pr : t.props) {
            step_done(pr.first->h);
            pr.first->last_prop_tick = s->tick;
        }
        {
            std::lock_guard<std::mutex> ls(s->mu_st);
            s->n_props += (long long)t.props.size();
            s->n_batched += 1;
            s->n_in_batches += (long long)t.props.size();
            s->cells += cells;
            s->host_batch_ms += ms_since(tb);
        }
        push_inflight(s, ev, MSG_ODO, std::move(arr), ev0, WORK_BATCH, bytes);
    }
    return true;
}

// The plain path: one loc_step per odometry message; a session's messages of the tick run on one
// pool stream (the next in turn, or the one its scan of the tick took).
bool launch_plain(loc_server s, TickWork& t) {
    const auto tp = std::chrono::steady_clock::now();
    SrvSession* prev = nullptr;
    for (auto& pm : t.plain) {                        // the plain path: one loc_step each
        SrvSession* ss = pm.first;
        if (ss != prev && ss->scan_tick != s->tick) {
            // a session's first message of the tick: the next stream in turn, unless the
            // session's scan of this tick already chose one (its steps follow the scan there)
            if (bind_stream(s, ss, (int)(s->plain_rr++ % s->pool.size())) != cudaSuccess) {
                set_failed(s, "stream ordering failed");
                return false;
            }
        }
        prev = ss;
        cudaEvent_t ev0 = get_event(s);
        if (!ev0 || cudaEventRecord(ev0, s->pool[(size_t)ss->stream_idx]) != cudaSuccess) {
            set_failed(s, "event record failed");
            return false;
        }
        const loc_status st = loc_step(ss->h, pm.second.u, pm.second.v, pm.second.w);
        if (st < 0) {
            set_failed(s, std::string("loc_step: ") + loc_last_error(ss->h));
            return false;
        }
        if (st == LOC_OK) {
            cudaEvent_t ev = get_event(s);
            if (!ev || cudaEventRecord(ev, s->pool[(size_t)ss->stream_idx]) != cudaSuccess) {
                set_failed(s, "event record failed");
                return false;
            }
            if (cudaEventRecord(ss->tail_ev, s->pool[(size_t)ss->stream_idx]) != cudaSuccess) {
                set_failed(s, "event record failed");
                return false;
            }
            ss->tail_valid = true;
            const double hw = (double)ss->p.H * ss->p.W;
            {
                std::lock_guard<std::mutex> ls(s->mu_st);
                s->n_props += 1;
                s->cells += hw * ss->p.K;
            }
            push_inflight(s, ev, MSG_ODO, std::vector<double>{pm.second.t_arr}, ev0, WORK_PLAIN,
                          hw * ss->p.K * 2.0 * (double)ss->h->elem + hw * 5.0);
        } else {
            {
                std::lock_guard<std::mutex> ls(s->mu_st);
                s->n_msgs += 1;
            }
            std::lock_guard<std::mutex> li(s->mu_inf);
            s->ev_free.push_back(ev0);                // nothing to time: the gate held the message
        }
    }
    if (!t.plain.empty()) {
        std::lock_guard<std::mutex> ls(s->mu_st);
        s->host_plain_ms += ms_since(tp);
    }
    return true;
}

// Scans first: a session's scan in this tick comes before its propagation in message order.
bool launch(loc_server s, TickWork& t) {
    if (!launch_scans(s, t) || !launch_batch(s, t) || !launch_plain(s, t)) return false;
    {
        std::lock_guard<std::mutex> ls(s->mu_st);
        s->n_msgs += t.absorbed;
        if (!t.props.empty() || !t.plain.empty() || !t.scans.empty()) s->n_ticks += 1;
    }
    s->tick += 1;
    return true;
}

void worker_main(loc_server s) {
    cudaSetDevice(s->device);
    for (;;) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            if (s->stop || s->failed) break;
        }
        if (!membership(s)) break;
        TickWork t;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            const auto tg = std::chrono::steady_clock::now();
            gather(s, t);
            if (!t.empty()) {
                std::lock_guard<std::mutex> ls(s->mu_st);
                s->host_gather_ms += ms_since(tg);
            }
            if (t.empty()) {
                s->busy = false;
                s->cv_done.notify_all();
                // sleep until a message, an admission or a close can make progress
                s->cv_work.wait_for(lk, std::chrono::milliseconds(2));
                continue;
            }
            s->busy = true;
        }
        const bool ok = launch(s, t);
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->busy = false;
            s->cv_done.notify_all();
        }
        if (!ok) break;
    }
}

}  // namespace

LOC_API void loc_server_params_default(loc_server_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->hbm_budget_bytes = 120e9;
    p->storage = LOC_BF16;
    p->batching = 1;
    p->tile = 0;
    p->use_graph = 1;
    p->n_streams = 32;
}

LOC_API loc_status loc_server_create(const loc_server_params* p, loc_server* out) {
    if (!out) return sfail(nullptr, LOC_ERR_INVALID_ARG, "out is null");
    *out = nullptr;
    if (!p) return sfail(nullptr, LOC_ERR_INVALID_ARG, "null params");
    if (!(p->hbm_budget_bytes > 0.0) || !std::isfinite(p->hbm_budget_bytes))
        return sfail(nullptr, LOC_ERR_INVALID_ARG, "hbm_budget_bytes must be finite and > 0");
    if (p->storage != LOC_F32 && p->storage != LOC_BF16 && p->storage != LOC_F16)
        return sfail(nullptr, LOC_ERR_INVALID_ARG, "unknown storage type");
    if (p->tile < 0 || p->tile > batch_num_cfgs())
        return sfail(nullptr, LOC_ERR_INVALID_ARG, "tile configuration out of range");
    if (p->n_streams < 1 || p->n_streams > 256) return sfail(nullptr, LOC_ERR_INVALID_ARG, "n_streams in [1, 256]");
    loc_server s = new (std::nothrow) loc_server_s();
    if (!s) return sfail(nullptr, LOC_ERR_OOM, "host allocation failed");
    s->prm = *p;
    s->t0 = std::chrono::steady_clock::now();
    cudaError_t e = cudaGetDevice(&s->device);
    for (int i = 0; i < p->n_streams && e == cudaSuccess; ++i) {
        cudaStream_t st = nullptr;
        e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e == cudaSuccess) s->pool.push_back(st);
    }
    for (int i = 0; i < kRing && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&s->ring[i], cudaEventDisableTiming);
    if (e != cudaSuccess) {
        const std::string m = std::string("loc_server_create: ") + cudaGetErrorString(e);
        for (cudaStream_t st : s->pool) cudaStreamDestroy(st);
        for (cudaEvent_t& ev : s->ring)
            if (ev) cudaEventDestroy(ev);
        delete s;
        return sfail(nullptr, LOC_ERR_CUDA, m);
    }
    for (size_t k = 1; k < kScanThreads; ++k) s->pool_threads.emplace_back(pool_main, s);
    s->worker = std::thread(worker_main, s);
    s->completer = std::thread(completer_main, s);
    *out = s;
    return LOC_OK;
}

LOC_API loc_status loc_server_open(loc_server s, const uint8_t* occ, const loc_params* p, int* id) {
    if (!s) return sfail(nullptr, LOC_ERR_INVALID_ARG, "null server");
    if (!occ || !p || !id) return sfail(s, LOC_ERR_INVALID_ARG, "null argument");
    loc_params q = *p;
    q.storage = s->prm.storage;
    q.stream = nullptr;
    size_t bytes = 0;
    if (loc_session_bytes(&q, &bytes) != LOC_OK) return sfail(s, LOC_ERR_INVALID_ARG, loc_last_error(nullptr));
    if (!(q.cell_m > 0.0) || !std::isfinite(q.cell_m)) return sfail(s, LOC_ERR_INVALID_ARG, "cell_m must be > 0");
    const size_t hw = (size_t)q.H * q.W;
    bool any_free = false;
    for (size_t i = 0; i < hw && !any_free; ++i) any_free = occ[i] == 0;
    if (!any_free) return sfail(s, LOC_ERR_INVALID_ARG, "map has no free cell");
    if ((double)bytes > s->prm.hbm_budget_bytes)
        return sfail(s, LOC_ERR_INVALID_ARG, "the session can never fit the memory budget");
    if (s->prm.batching) {
        if (q.kernel == LOC_KERNEL_GENERIC || (q.sigma_cross_cells > 0.0 && q.sigma_cross_cells != q.sigma_xy_cells) ||
            !step_tiled_eligible(q.H, q.W, q.K, radius(q.sigma_xy_cells, q.r_xy), radius(q.sigma_theta_bins, q.r_theta),
                                 q.storage))
            return sfail(s, LOC_ERR_INVALID_ARG, "a batched server needs sessions the tiled kernel can take");
    }
    SrvSession* ss = new (std::nothrow) SrvSession();
    if (!ss) return sfail(s, LOC_ERR_OOM, "host allocation failed");
    ss->occ.assign(occ, occ + hw);
    ss->p = q;
    ss->bytes = bytes;
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->failed) {
        delete ss;
        set_thread_error(("server failed: " + s->err).c_str());
        return LOC_ERR_STATE;
    }
    ss->id = (int)s->sessions.size();
    ss->stream_idx = ss->id % (int)s->pool.size();
    s->sessions.push_back(ss);
    s->admit_q.push_back(ss->id);
    *id = ss->id;
    s->cv_work.notify_one();
    return LOC_OK;
}

LOC_API loc_status loc_server_close(loc_server s, int id) {
    if (!s) return sfail(nullptr, LOC_ERR_INVALID_ARG, "null server");
    std::lock_guard<std::mutex> lk(s->mu);
    if (id < 0 || (size_t)id >= s->sessions.size()) {
        set_thread_error("unknown session id");
        return LOC_ERR_INVALID_ARG;
    }
    s->sessions[(size_t)id]->closing = true;
    s->cv_work.notify_one();
    return LOC_OK;
}

LOC_API loc_status loc_server_odometry(loc_server s, int n, const int* ids, const double* u, const double* v,
                                       const double* w, const double* t_arrival) {
    if (!s) return sfail(nullptr, LOC_ERR_INVALID_ARG, "null server");
    if (n < 0 || (n > 0 && (!ids || !u || !v || !w))) return sfail(s, LOC_ERR_INVALID_ARG, "null arrays");
    const double now = s->now();
    double first = -1.0;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->failed) {
            set_thread_error(("server failed: " + s->err).c_str());
            return LOC_ERR_STATE;
        }
        for (int i = 0; i < n; ++i) {
            if (ids[i] < 0 || (size_t)ids[i] >= s->sessions.size() || s->sessions[(size_t)ids[i]]->closing ||
                s->sessions[(size_t)ids[i]]->state >= LOC_SESSION_CLOSED) {
                set_thread_error("unknown, closed or failed session id");
                return LOC_ERR_INVALID_ARG;
            }
            if (!std::isfinite(u[i]) || !std::isfinite(v[i]) || !std::isfinite(w[i]) ||
                (t_arrival && !std::isfinite(t_arrival[i]))) {
                set_thread_error("odometry and arrival times must be finite");
                return LOC_ERR_INVALID_ARG;
            }
        }
        for (int i = 0; i < n; ++i) {
            SrvMsg m;
            m.kind = MSG_ODO;
            m.u = u[i];
            m.v = v[i];
            m.w = w[i];
            m.t_arr = t_arrival ? t_arrival[i] : now;
            if (first < 0.0 || m.t_arr < first) first = m.t_arr;
            s->sessions[(size_t)ids[i]]->q.push_back(m);
        }
        s->cv_work.notify_one();
    }
    if (n > 0) note_arrival(s, first);
    return LOC_OK;
}

LOC_API loc_status loc_server_scan(loc_server s, int id, const float* ranges, int n_beams, double angle_min,
                                   double angle_inc, double r_max, int beam_stride, double sigma_r, double t_arrival) {
    if (!s) return sfail(nullptr, LOC_ERR_INVALID_ARG, "null server");
    if (!ranges || n_beams <= 0 || beam_stride < 1 || !std::isfinite(angle_min) || !std::isfinite(angle_inc) ||
        !(r_max > 0.0) || !std::isfinite(r_max) || !(sigma_r > 0.0) || !std::isfinite(sigma_r) ||
        !std::isfinite(t_arrival))
        return sfail(s, LOC_ERR_INVALID_ARG, "scan: ranges, n_beams > 0, stride >= 1, finite angles, r_max, sigma_r > 0");
    for (int b = 0; b < n_beams; ++b)
        if (!std::isfinite(ranges[b]) || ranges[b] < 0.0f)
            return sfail(s, LOC_ERR_INVALID_ARG, "ranges must be finite and >= 0");
    SrvScan* sc = new (std::nothrow) SrvScan();
    if (!sc) return sfail(s, LOC_ERR_OOM, "host allocation failed");
    sc->ranges.assign(ranges, ranges + n_beams);
    sc->angle_min = angle_min;
    sc->angle_inc = angle_inc;
    sc->r_max = r_max;
    sc->sigma_r = sigma_r;
    sc->stride = beam_stride;
    SrvMsg m;
    m.kind = MSG_SCAN;
    m.scan = sc;
    m.t_arr = t_arrival < 0.0 ? s->now() : t_arrival;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->failed || id < 0 || (size_t)id >= s->sessions.size() || s->sessions[(size_t)id]->closing ||
            s->sessions[(size_t)id]->state >= LOC_SESSION_CLOSED) {
            delete sc;
            set_thread_error(s->failed ? "server failed" : "unknown, closed or failed session id");
            return s->failed ? LOC_ERR_STATE : LOC_ERR_INVALID_ARG;
        }
        s->sessions[(size_t)id]->q.push_back(m);
        s->cv_work.notify_one();
    }
    note_arrival(s, m.t_arr);
    return LOC_OK;
}

LOC_API double loc_server_now(loc_server s) { return s ? s->now() : 0.0; }

LOC_API loc_status loc_server_drain(loc_server s, double timeout_s) {
    if (!s) return sfail(nullptr, LOC_ERR_INVALID_ARG, "null server");
    const auto until = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        if (s->failed) {
            set_thread_error(("server failed: " + s->err).c_str());
            return LOC_ERR_STATE;
        }
        bool idle = !s->busy;
        for (SrvSession* ss : s->sessions)
            if (ss->state == LOC_SESSION_ACTIVE && !ss->q.empty()) idle = false;
        for (SrvSession* ss : s->sessions)          // sessions closing or admissible change the set
            if (ss->state == LOC_SESSION_ACTIVE && ss->closing) idle = false;
        if (!s->admit_q.empty()) {
            const SrvSession* head = s->sessions[(size_t)s->admit_q.front()];
            if (head->closing || (double)(s->used_bytes + head->bytes) <= s->prm.hbm_budget_bytes) idle = false;
        }
        if (idle) {
            std::lock_guard<std::mutex> li(s->mu_inf);
            idle = s->inflight.empty();
        }
        if (idle) return LOC_OK;
        if (std::chrono::steady_clock::now() >= until) {
            set_thread_error("loc_server_drain timed out");
            return LOC_ERR_TIMEOUT;
        }
        s->cv_work.notify_one();
        s->cv_done.wait_for(lk, std::chrono::milliseconds(1));
    }
}

LOC_API loc_status loc_server_stats(loc_server s, loc_server_stats_t* o) {
    if (!s || !o) return sfail(s, LOC_ERR_INVALID_ARG, "null argument");
    std::memset(o, 0, sizeof(*o));
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (SrvSession* ss : s->sessions) {
            o->n_pending += ss->state == LOC_SESSION_PENDING;
            o->n_active += ss->state == LOC_SESSION_ACTIVE;
            o->n_closed += ss->state == LOC_SESSION_CLOSED;
            o->n_failed += ss->state == LOC_SESSION_FAILED;
        }
        o->bytes_used = (double)s->used_bytes;
        o->bytes_budget = s->prm.hbm_budget_bytes;
    }
    std::vector<double> a, b;
    {
        std::lock_guard<std::mutex> ls(s->mu_st);
        o->n_ticks = s->n_ticks;
        o->n_messages = s->n_msgs;
        o->n_propagations = s->n_props;
        o->n_scans = s->n_scans;
        o->cell_updates = s->cells;
        o->mean_batch = s->n_batched ? (double)s->n_in_batches / (double)s->n_batched : 0.0;
        o->first_s = s->first_s;
        o->last_s = s->last_s;
        o->batch_device_ms = s->dev_ms[WORK_BATCH];
        o->batch_alg_bytes = s->dev_bytes[WORK_BATCH];
        o->n_batches = s->dev_n[WORK_BATCH];
        o->scan_device_ms = s->dev_ms[WORK_SCAN];
        o->n_scans_timed = s->dev_n[WORK_SCAN];
        o->plain_device_ms = s->dev_ms[WORK_PLAIN];
        o->plain_alg_bytes = s->dev_bytes[WORK_PLAIN];
        o->n_plain = s->dev_n[WORK_PLAIN];
        o->host_gather_ms = s->host_gather_ms;
        o->host_batch_ms = s->host_batch_ms;
        o->host_scan_ms = s->host_scan_ms;
        o->host_plain_ms = s->host_plain_ms;
        a = s->lat_step;
        b = s->lat_scan;
    }
    o->step_p50_ms = pct(a, 0.50);
    o->step_p99_ms = pct(a, 0.99);
    o->step_max_ms = a.empty() ? 0.0 : *std::max_element(a.begin(), a.end());
    o->scan_p50_ms = pct(b, 0.50);
    o->scan_p99_ms = pct(b, 0.99);
    o->scan_max_ms = b.empty() ? 0.0 : *std::max_element(b.begin(), b.end());
    return LOC_OK;
}

LOC_API loc_status loc_server_reset_stats(loc_server s) {
    if (!s) return sfail(nullptr, LOC_ERR_INVALID_ARG, "null server");
    std::lock_guard<std::mutex> ls(s->mu_st);
    s->lat_step.clear();
    s->lat_scan.clear();
    s->n_ticks = s->n_msgs = s->n_props = s->n_scans = s->n_batched = s->n_in_batches = 0;
    s->cells = 0.0;
    s->first_s = -1.0;
    s->last_s = 0.0;
    for (int w = 0; w < 3; ++w) {
        s->dev_ms[w] = s->dev_bytes[w] = 0.0;
        s->dev_n[w] = 0;
    }
    s->host_gather_ms = s->host_batch_ms = s->host_scan_ms = s->host_plain_ms = 0.0;
    return LOC_OK;
}

LOC_API loc_status loc_server_session(loc_server s, int id, int* state, loc_handle* h) {
    if (!s) return sfail(nullptr, LOC_ERR_INVALID_ARG, "null server");
    std::lock_guard<std::mutex> lk(s->mu);
    if (id < 0 || (size_t)id >= s->sessions.size()) {
        set_thread_error("unknown session id");
        return LOC_ERR_INVALID_ARG;
    }
    SrvSession* ss = s->sessions[(size_t)id];
    if (state) *state = ss->state;
    if (h) *h = ss->state == LOC_SESSION_ACTIVE ? ss->h : nullptr;
    return LOC_OK;
}

LOC_API loc_status loc_server_destroy(loc_server s) {
    if (!s) return LOC_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv_work.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    {
        std::lock_guard<std::mutex> lk(s->mu_pool);
        s->pool_stop = true;
    }
    s->cv_pool.notify_all();
    for (std::thread& th : s->pool_threads)
        if (th.joinable()) th.join();
    s->stop_completer = true;
    if (s->completer.joinable()) s->completer.join();
    sync_all(s);
    if (s->core_live) batch_release(&s->core);
    for (SrvSession* ss : s->sessions) {
        for (SrvMsg& m : ss->q) delete m.scan;
        if (ss->h) loc_destroy(ss->h);
        if (ss->scan_ev) cudaEventDestroy(ss->scan_ev);
        if (ss->tail_ev) cudaEventDestroy(ss->tail_ev);
        delete ss;
    }
    for (cudaEvent_t ev : s->ev_free) cudaEventDestroy(ev);
    for (cudaEvent_t ev : s->ring) cudaEventDestroy(ev);
    for (cudaStream_t st : s->pool) cudaStreamDestroy(st);
    delete s;
    return LOC_OK;
}

LOC_API const char* loc_server_last_error(loc_server s) { return s ? s->err.c_str() : ""; }
