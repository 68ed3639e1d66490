// The session object behind loc_handle and the host helpers shared by the C-ABI files
// (single-session calls, the batched launch and the serving loop).  Internal to the library.
#pragma once

#include <string>
#include <vector>

#include "kernels.h"
#include "loc.h"

struct loc_session {
    loc_params p{};
    int r_xy = 0, r_th = 0;
    float gx[2 * LOC_MAX_R_XY + 1]{};
    float gt[2 * LOC_MAX_R_THETA + 1]{};
    cudaStream_t stream = nullptr;
    int device = 0;
    size_t elem = 4;               // bytes per stored belief value
    size_t hw = 0, n = 0;          // H*W, K*H*W
    long long n_free = 0;
    float inv_uniform = 0.0f;
    // device buffers
    void* B[2] = {nullptr, nullptr};
    int cur = 0;                   // B[cur] holds the current stored tensor
    uint8_t* trav = nullptr;
    float* corr = nullptr;
    loc::SessionDev* sd = nullptr;
    unsigned long long reinit_reported = 0;   // restart count last reported as LOC_WARN_REINIT
    double* partials = nullptr;
    unsigned int nparts = 0;
    // the argmax fused into the tiled propagation: per-CTA candidates, and whether the result
    // in argmax_idx / argmax_val belongs to the current tensor (set by loc_step, cleared by
    // every other change of the tensor)
    float* am_pv = nullptr;
    long long* am_pi = nullptr;
    bool am_valid = false;
    void* argmax_scratch = nullptr;
    long long* argmax_idx = nullptr;
    float* argmax_val = nullptr;
    unsigned char* pinned = nullptr;   // 64 bytes of pinned host memory for small readbacks
    loc::EstimateOut* est = nullptr;   // loc_estimate's device results (allocated on first use)
    // LIDAR sample update scratch (allocated on first use)
    bool lidar_ready = false;
    int cap = 0;                   // capacity of the sample list
    float* m = nullptr;            // belief map [H][W]
    uint32_t* travbits = nullptr;  // the map as bits [H][ceil(W / 32)] (the ray casts' window)
    uint8_t* sel = nullptr;        // selection mask [H][W]
    int* rowcnt = nullptr;         // per-row selections [H]
    int* rowoff = nullptr;         // exclusive prefix [H]
    float* bnd = nullptr;          // row-block boundary rows for the dithering wavefront
    int* prog = nullptr;           // their progress counters
    int32_t* samples = nullptr;    // sampled cells [cap]
    float* logL = nullptr;         // log-likelihood [cap][K]
    int* dscal = nullptr;          // device scalars: count, maxL (as uint), fs (as float)
    void* rs = nullptr;            // reweight scalars
    float* dirs = nullptr;         // distinct beam directions (cos, sin) [cap_dirs][2]
    int32_t* dir_of = nullptr;     // direction of (bin, used beam) [K][cap_beams]
    float* z = nullptr;            // used ranges [cap_beams]
    int cap_dirs = 0, cap_beams = 0, cap_dir_of = 0;
    // pinned staging of the scan tables (two slots; a slot is reused once the copies that
    // read it, marked by its event, have run)
    unsigned char* scan_pin[2] = {nullptr, nullptr};
    size_t scan_pin_cap[2] = {0, 0};
    cudaEvent_t scan_pin_ev[2] = {nullptr, nullptr};
    int scan_slot = 0;
    long long n_lidar = 0;
    // dense scan update (allocated by loc_range_table / the first dense update)
    uint8_t* table = nullptr;      // expected-range codes [table_A][H][W]
    int table_A = 0;
    double table_rmax = 0.0;
    float* dense_logL = nullptr;   // log-likelihood of every state [K][H][W]
    int* dense_m = nullptr;        // table offsets of the used beams [cap_dense]
    float* dense_z = nullptr;      // their ranges over the code step [cap_dense]
    unsigned int* dense_max = nullptr;
    int cap_dense = 0, cap_dense_z = 0;
    long long n_dense = 0;
    bool aniso = false;            // anisotropic motion noise (step_aniso.cu)
    bool aniso_tma = false;        // ... with its input boxes by TMA (tmap holds its maps)
    bool tiled = false;            // use the TMA-tiled kernel
    int tile_cfg = 0;              // its tile configuration
    unsigned char tmap[2][128] __attribute__((aligned(128)));   // tensor maps of B[0], B[1]
    // host-side state (FP64)
    double theta = 0.0, px = 0.0, py = 0.0;
    long long n_prop = 0;
    bool failed = false;
    std::string err;
    std::vector<void*> owned;
};


namespace loc {

loc_status fail(loc_session* s, loc_status code, const std::string& msg);
loc_status cuda_fail(loc_session* s, cudaError_t e, const char* what);
void* dev_alloc(loc_session* s, size_t bytes);
void release_all(loc_session* s);
loc_status check_live(loc_session* h);
// Kernel radius for sigma (given >= 0 overrides), as loc_create derives it.
int radius(double sigma, int given);
// Synchronise the session's stream and turn device-side error flags into a status.
loc_status sync_and_check(loc_session* h);
// The status for device-side error flags already read back.
loc_status check_status(loc_session* h, int status);

// Odometry bookkeeping of Section III-A (Eq. 2-3): accumulate an increment and report whether
// the gate lets a propagation through; the per-bin shift table of the accumulated
// translation; and the bookkeeping after a propagation was enqueued (ping-pong flip,
// translation reset, counter).
bool odometry_advance(loc_session* h, double u, double v, double w);
void shift_table(const loc_session* h, Shift* sh);
void step_done(loc_session* h);

}  // namespace loc
