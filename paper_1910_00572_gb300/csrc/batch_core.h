// Host side of the batched launch, shared by the batch C-ABI and the serving loop (internal).
//
// A BatchCore owns the device tables of one fixed group of sessions: the per-session
// constants (uploaded once), the per-tick table (copied from one of two pinned host buffers
// every tick) and the launch control words; it runs on a stream of its own and can capture
// the tick in two CUDA graphs, one per pinned buffer.
#pragma once

#include <vector>

#include "session.h"

namespace loc {

struct BatchCore {
    std::vector<loc_session*> sess;
    std::vector<int> ntiles;               // tiles of each session in the current configuration
    std::vector<int> order;                // sessions by decreasing K (work order of a tick)
    std::vector<int> sh_off;               // first shift-table entry of each session
    int storage = LOC_F32;
    cudaStream_t user = nullptr;           // the sessions' stream
    cudaStream_t bs = nullptr;             // the batch's own stream (capturable)
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    int cfg = 0, grid = 0;
    float tune_ms[8] = {};
    long long tiles_all = 0;               // tiles of all sessions
    BatchLayout lay{};
    BatchStatic* d_static = nullptr;
    void* d_tick = nullptr;
    void* h_tick[2] = {nullptr, nullptr};  // pinned, used by alternate ticks
    cudaEvent_t done[2] = {nullptr, nullptr};
    BatchCtl* d_ctl = nullptr;
    bool use_graph = false;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int parity = 0;
    long long n_ticks = 0;
};

// Check that the sessions can share one launch (distinct, live, tiled-eligible, one storage
// type, stream and device); returns "" or the reason.
std::string batch_check(loc_session* const* sessions, int n);
// Allocate and fill the tables; tile 0 runs the autotuner (dry runs that change no session).
cudaError_t batch_init(BatchCore* c, loc_session* const* sessions, int n, int tile, bool use_graph);
void batch_release(BatchCore* c);
// Begin a tick: wait until the pinned buffer of this tick is free again (its copy two ticks
// ago has run) and return its per-session headers and shift tables (session s owns K_s
// entries from shift_slot(c, s)).
cudaError_t batch_begin(BatchCore* c, BatchTick** hdr, Shift** shifts);
Shift* batch_shift_slot(BatchCore* c, Shift* shifts, int s);
// Launch the tick for the sessions flagged in active[] (headers and shift tables filled by
// the caller); records `done` (may be null) after the tick's work.  With join_user the launch
// is ordered after the earlier work of the sessions' stream and that stream's later work after
// it; without, the caller orders it.  Does nothing when no session is active.
cudaError_t batch_launch(BatchCore* c, const std::vector<char>& active, cudaEvent_t done, bool join_user);

}  // namespace loc
