// C-ABI of the localizer: session state on the host, device buffers, odometry bookkeeping
// (Section III-A, Eq. 2, the Alg. 1 gate) and the launches of the device kernels.
#include <algorithm>
#include <climits>
#include <cstddef>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "session.h"

#define LOC_API extern "C" __attribute__((visibility("default")))

using namespace loc;

namespace {

thread_local std::string g_thread_err;
loc_alloc_fn g_alloc = nullptr;
loc_free_fn g_free = nullptr;
void* g_alloc_ctx = nullptr;

}  // namespace

void loc::set_thread_error(const char* msg) { g_thread_err = msg ? msg : ""; }

namespace loc {

loc_status fail(loc_session* s, loc_status code, const std::string& msg) {
    if (s) {
        s->err = msg;
        if (code == LOC_ERR_CUDA || code == LOC_ERR_TIMEOUT) s->failed = true;
    } else {
        g_thread_err = msg;
    }
    return code;
}

loc_status cuda_fail(loc_session* s, cudaError_t e, const char* what) {
    return fail(s, LOC_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

void* dev_alloc(loc_session* s, size_t bytes) {
    void* p = nullptr;
    if (g_alloc) {
        p = g_alloc(bytes, (void*)s->stream, g_alloc_ctx);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) s->owned.push_back(p);
    return p;
}

void release_all(loc_session* s) {
    if (s->pinned) cudaFreeHost(s->pinned);
    s->pinned = nullptr;
    for (int k = 0; k < 2; ++k) {
        if (s->scan_pin_ev[k]) {
            cudaEventSynchronize(s->scan_pin_ev[k]);
            cudaEventDestroy(s->scan_pin_ev[k]);
        }
        if (s->scan_pin[k]) cudaFreeHost(s->scan_pin[k]);
        s->scan_pin[k] = nullptr;
        s->scan_pin_ev[k] = nullptr;
    }
    for (void* p : s->owned) {
        if (g_free) g_free(p, (void*)s->stream, g_alloc_ctx);
        else cudaFree(p);
    }
    s->owned.clear();
}

void taps(double sigma, int r, float* out) {
    if (r == 0 || sigma <= 0.0) {
        for (int d = 0; d <= 2 * r; ++d) out[d] = d == r ? 1.0f : 0.0f;
        return;
    }
    double g[2 * 8 + 1], sum = 0.0;
    for (int d = -r; d <= r; ++d) {
        g[d + r] = std::exp(-0.5 * (d / sigma) * (d / sigma));
        sum += g[d + r];
    }
    for (int d = 0; d <= 2 * r; ++d) out[d] = (float)(g[d] / sum);
}

// Kernel radius: the given one, else ceil(3 sigma).  A sigma that is not finite, or whose
// radius would exceed every supported maximum, gives INT_MAX (rejected by the callers' radius
// checks) without converting an out-of-range double to int.
int radius(double sigma, int given) {
    if (given >= 0) return given;
    if (std::isnan(sigma) || !(3.0 * sigma <= 1024.0)) return INT_MAX;
    return sigma <= 0.0 ? 0 : (int)std::ceil(3.0 * sigma);
}

loc_status check_live(loc_session* h) {
    if (!h) return fail(nullptr, LOC_ERR_INVALID_ARG, "null handle");
    if (h->failed) return fail(h, LOC_ERR_STATE, "handle failed earlier: " + h->err);
    return LOC_OK;
}

loc_status sync_and_check(loc_session* h) {
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamSynchronize");
    // the device status and the restart count are adjacent in SessionDev: one copy
    struct {
        int status, pad;
        unsigned long long n_reinit;
    } d{};
    static_assert(offsetof(SessionDev, n_reinit) == offsetof(SessionDev, status) + 8, "SessionDev layout");
    e = cudaMemcpy(&d, &h->sd->status, sizeof(d), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemcpy(status)");
    const loc_status st = check_status(h, d.status);
    if (st != LOC_OK) return st;
    if (d.n_reinit > h->reinit_reported) {         // restarts since the last report
        h->reinit_reported = d.n_reinit;
        return LOC_WARN_REINIT;
    }
    return LOC_OK;
}

loc_status check_status(loc_session* h, int status) {
    if (status & LOC_DEV_ERR_TIMEOUT) return fail(h, LOC_ERR_TIMEOUT, "device wait timed out");
    if (status & LOC_DEV_ERR_NONFINITE_Z) {
        h->failed = true;
        return fail(h, LOC_ERR_STATE, "normaliser was not finite");
    }
    return LOC_OK;
}

}  // namespace loc

LOC_API void loc_params_default(loc_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->sigma_xy_cells = 0.5;
    p->sigma_theta_bins = 1.0;
    p->r_xy = -1;
    p->r_theta = -1;
    p->min_shift_cells = 0.0;
    p->storage = LOC_F32;
    p->n_samples = 4096;
    p->stream = nullptr;
    p->kernel = LOC_KERNEL_AUTO;
    p->tile = 0;
    p->sigma_cross_cells = 0.0;
}

LOC_API void loc_set_allocator(loc_alloc_fn alloc, loc_free_fn release, void* ctx) {
    g_alloc = (alloc && release) ? alloc : nullptr;
    g_free = (alloc && release) ? release : nullptr;
    g_alloc_ctx = (alloc && release) ? ctx : nullptr;
}

LOC_API loc_status loc_session_bytes(const loc_params* p, size_t* bytes) {
    if (!p || !bytes) return fail(nullptr, LOC_ERR_INVALID_ARG, "null argument");
    if (p->H <= 0 || p->W <= 0 || p->K <= 0 || p->K > LOC_MAX_K || p->n_samples < 0)
        return fail(nullptr, LOC_ERR_INVALID_ARG, "H, W must be > 0, 0 < K <= LOC_MAX_K, n_samples >= 0");
    if (p->storage != LOC_F32 && p->storage != LOC_BF16 && p->storage != LOC_F16)
        return fail(nullptr, LOC_ERR_INVALID_ARG, "unknown storage type");
    // every allocation rounded up to 512 bytes, as the device allocators hand them out
    auto r = [](size_t b) { return (b + 511) & ~(size_t)511; };
    const size_t H = (size_t)p->H, W = (size_t)p->W, K = (size_t)p->K, hw = H * W, n = hw * K;
    const size_t elem = p->storage == LOC_F32 ? 4 : 2;
    size_t nparts = step_num_blocks(p->H, p->W);
    if (nparts < 4096) nparts = 4096;
    size_t b = 2 * r(n * elem) + r(hw) + r(hw * 4) + r(sizeof(SessionDev)) + r(nparts * 8) +
               r(nparts * 12) + r(argmax_scratch_bytes(n)) + r(16);
    // LIDAR scratch (allocated by the first scan update); the scan tables are sized for a
    // 1080-beam scan
    size_t cap = 2 * (size_t)p->n_samples + 4 * (H + W) + 1024;
    if (cap > hw) cap = hw;
    const size_t nrb = (H + 31) / 32;
    b += r(hw * 4) + r(hw) + 2 * r(H * 4) + r((nrb + 1) * W * 4) + r((nrb + 2) * 4) + r(cap * 4) +
         r(cap * K * 4) + r(64) + r(reweight_scalars_bytes()) + r(K * 1080 * 8) + r(1080 * 4) + r(K * 1080 * 4) +
         r(H * ((W + 31) / 32) * 4);
    *bytes = b;
    return LOC_OK;
}

LOC_API loc_status loc_create(const uint8_t* occ, const loc_params* p, loc_handle* out) {
    if (!out) return fail(nullptr, LOC_ERR_INVALID_ARG, "out is null");
    *out = nullptr;
    if (!occ || !p) return fail(nullptr, LOC_ERR_INVALID_ARG, "null map or params");
    if (p->H <= 0 || p->W <= 0 || p->K <= 0 || p->K > LOC_MAX_K)
        return fail(nullptr, LOC_ERR_INVALID_ARG, "H, W must be > 0 and 0 < K <= LOC_MAX_K");
    if (!(p->cell_m > 0.0) || !std::isfinite(p->cell_m))
        return fail(nullptr, LOC_ERR_INVALID_ARG, "cell_m must be finite and > 0");
    if (!(p->sigma_xy_cells >= 0.0) || !(p->sigma_theta_bins >= 0.0) ||
        !std::isfinite(p->sigma_xy_cells) || !std::isfinite(p->sigma_theta_bins))
        return fail(nullptr, LOC_ERR_INVALID_ARG, "sigmas must be finite and >= 0");
    if (p->storage != LOC_F32 && p->storage != LOC_BF16 && p->storage != LOC_F16)
        return fail(nullptr, LOC_ERR_INVALID_ARG, "unknown storage type");
    if (!(p->min_shift_cells >= 0.0) || !std::isfinite(p->min_shift_cells))
        return fail(nullptr, LOC_ERR_INVALID_ARG, "min_shift_cells must be finite and >= 0");
    if (!(p->sigma_cross_cells >= 0.0) || !std::isfinite(p->sigma_cross_cells))
        return fail(nullptr, LOC_ERR_INVALID_ARG, "sigma_cross_cells must be finite and >= 0");
    // Eq. 6 with sigma_x != sigma_y: the x/y kernel of each bin is rotated to its heading
    const bool aniso = p->sigma_cross_cells > 0.0 && p->sigma_cross_cells != p->sigma_xy_cells;
    if (aniso && !(p->sigma_xy_cells > 0.0))
        return fail(nullptr, LOC_ERR_INVALID_ARG, "anisotropic noise needs sigma_xy_cells > 0");
    const int rxy = radius(aniso ? std::max(p->sigma_xy_cells, p->sigma_cross_cells) : p->sigma_xy_cells, p->r_xy);
    const int rth = radius(p->sigma_theta_bins, p->r_theta);
    if (rxy > LOC_MAX_R_XY || rth > LOC_MAX_R_THETA)
        return fail(nullptr, LOC_ERR_INVALID_ARG, "kernel radius above LOC_MAX_R_XY / LOC_MAX_R_THETA");
    if (p->n_samples < 0) return fail(nullptr, LOC_ERR_INVALID_ARG, "n_samples must be >= 0");
    if (p->kernel < LOC_KERNEL_AUTO || p->kernel > LOC_KERNEL_TILED)
        return fail(nullptr, LOC_ERR_INVALID_ARG, "unknown kernel selection");
    if (aniso && p->kernel == LOC_KERNEL_TILED)
        return fail(nullptr, LOC_ERR_INVALID_ARG, "anisotropic noise runs on the generic kernel path");
    const bool tiled_ok = !aniso && step_tiled_eligible(p->H, p->W, p->K, rxy, rth, p->storage);
    if (p->tile < 0 || p->tile > step_tiled_num_cfgs())
        return fail(nullptr, LOC_ERR_INVALID_ARG, "tile configuration out of range");
    if (p->kernel == LOC_KERNEL_TILED && !tiled_ok)
        return fail(nullptr, LOC_ERR_INVALID_ARG, "the tiled kernel needs radii 2/3, K >= 8 and aligned W");

    const size_t hw = (size_t)p->H * p->W;
    std::vector<uint8_t> trav(hw);
    long long n_free = 0;
    for (size_t q = 0; q < hw; ++q) {
        trav[q] = occ[q] == 0 ? 1 : 0;
        n_free += trav[q];
    }
    if (n_free == 0) return fail(nullptr, LOC_ERR_INVALID_ARG, "map has no free cell");

    loc_session* s = new (std::nothrow) loc_session();
    if (!s) return fail(nullptr, LOC_ERR_OOM, "host allocation failed");
    s->p = *p;
    s->aniso = aniso;
    s->r_xy = rxy;
    s->r_th = rth;
    taps(p->sigma_xy_cells, rxy, s->gx);
    taps(p->sigma_theta_bins, rth, s->gt);
    s->stream = (cudaStream_t)p->stream;
    cudaGetDevice(&s->device);
    s->elem = p->storage == LOC_F32 ? 4 : 2;
    s->hw = hw;
    s->n = hw * (size_t)p->K;
    s->n_free = n_free;
    s->inv_uniform = (float)(1.0 / ((double)p->K * (double)n_free));
    s->nparts = step_num_blocks(p->H, p->W);
    if (s->nparts < 4096) s->nparts = 4096;

    s->B[0] = dev_alloc(s, s->n * s->elem);
    s->B[1] = dev_alloc(s, s->n * s->elem);
    s->trav = (uint8_t*)dev_alloc(s, hw);
    s->corr = (float*)dev_alloc(s, hw * sizeof(float));
    s->sd = (SessionDev*)dev_alloc(s, sizeof(SessionDev));
    s->partials = (double*)dev_alloc(s, s->nparts * sizeof(double));
    s->am_pi = (long long*)dev_alloc(s, s->nparts * (sizeof(long long) + sizeof(float)));
    s->am_pv = s->am_pi ? (float*)(s->am_pi + s->nparts) : nullptr;
    s->argmax_scratch = dev_alloc(s, argmax_scratch_bytes(s->n));
    s->argmax_idx = (long long*)dev_alloc(s, sizeof(long long) + sizeof(float));
    if (!s->B[0] || !s->B[1] || !s->trav || !s->corr || !s->sd || !s->partials || !s->am_pi ||
        !s->argmax_scratch || !s->argmax_idx) {
        release_all(s);
        delete s;
        return fail(nullptr, LOC_ERR_OOM, "device allocation failed");
    }
    s->argmax_val = (float*)(s->argmax_idx + 1);
    if (cudaMallocHost(&s->pinned, 64) != cudaSuccess) {
        cudaGetLastError();
        release_all(s);
        delete s;
        return fail(nullptr, LOC_ERR_OOM, "pinned host allocation failed");
    }
    s->tiled = tiled_ok && p->kernel != LOC_KERNEL_GENERIC;
    if (aniso && aniso_tma_eligible(p->W, p->storage)) {
        s->aniso_tma = true;
        for (int b = 0; b < 2; ++b) {
            if (make_aniso_tmap(s->tmap[b], s->B[b], p->storage, p->H, p->W, p->K, rxy) != cudaSuccess) {
                release_all(s);
                delete s;
                return fail(nullptr, LOC_ERR_CUDA, "cuTensorMapEncodeTiled failed");
            }
        }
    }
    if (s->tiled) {
        s->tile_cfg = p->tile > 0 ? p->tile : step_tiled_default_cfg(p->H, p->W, p->K, p->storage);
        for (int b = 0; b < 2; ++b) {
            if (make_step_tmap(s->tmap[b], s->B[b], p->storage, p->H, p->W, p->K, s->tile_cfg) != cudaSuccess) {
                release_all(s);
                delete s;
                return fail(nullptr, LOC_ERR_CUDA, "cuTensorMapEncodeTiled failed");
            }
        }
    }

    SessionDev init{};
    init.Z = 1.0;
    init.inv_Z = 1.0f;
    init.reinit = 1;               // the stored tensor reads as uniform over free cells
    cudaError_t e = cudaMemcpyAsync(s->trav, trav.data(), hw, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess)   // the argmax pass's arrival counter starts at zero
        e = cudaMemsetAsync(s->argmax_scratch, 0, argmax_scratch_bytes(s->n), s->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->sd, &init, sizeof(init), cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = launch_edge_correction(s->trav, s->corr, p->H, p->W, s->gx, rxy, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) {
        std::string msg = std::string("loc_create: ") + cudaGetErrorString(e);
        release_all(s);
        delete s;
        return fail(nullptr, LOC_ERR_CUDA, msg);
    }
    *out = s;
    return LOC_OK;
}

namespace loc {

// Section III-A / Eq. 2: accumulate the odometry increment (translate in the frame of
// theta_{t-1}, then rotate).  Returns whether the gate lets a propagation through.
bool odometry_advance(loc_session* h, double u, double v, double w) {
    const double c = std::cos(h->theta), s = std::sin(h->theta);
    h->px += c * u - s * v;
    h->py += s * u + c * v;
    h->theta += w;
    return std::hypot(h->px, h->py) / h->p.cell_m >= h->p.min_shift_cells;
}

// Eq. 2-3: the per-bin source offsets of the accumulated translation.
void shift_table(const loc_session* h, Shift* sh) {
    const double cell = h->p.cell_m;
    const int K = h->p.K;
    for (int k = 0; k < K; ++k) {
        const double ang = 2.0 * M_PI * k / K;
        const double ck = std::cos(ang), sk = std::sin(ang);
        const double sx = (ck * h->px - sk * h->py) / cell;   // R(k dTheta) p, in cells
        const double sy = (sk * h->px + ck * h->py) / cell;
        // pull source: integer part and fraction of -s.  A fraction within 1e-9 of a whole
        // cell (e.g. 3 cos(pi/2) = 1.8e-16) is snapped, which changes the result by under
        // 1e-9 relative and keeps integer shifts exact permutations.
        double ox = std::floor(-sx), oy = std::floor(-sy);
        double fx = -sx - ox, fy = -sy - oy;
        if (fx < 1e-9) fx = 0.0;
        if (fx > 1.0 - 1e-9) { fx = 0.0; ox += 1.0; }
        if (fy < 1e-9) fy = 0.0;
        if (fy > 1.0 - 1e-9) { fy = 0.0; oy += 1.0; }
        sh[k].ox = (int)ox;
        sh[k].oy = (int)oy;
        sh[k].fx = (float)fx;
        sh[k].fy = (float)fy;
    }
}

// After a propagation was enqueued: the output buffer becomes current.  A fused argmax
// result, if any, is for the previous tensor (loc_step marks a fresh one afterwards).
void step_done(loc_session* h) {
    h->cur = 1 - h->cur;
    h->px = h->py = 0.0;
    h->n_prop += 1;
    h->am_valid = false;
}

}  // namespace loc

LOC_API loc_status loc_step(loc_handle h, double u, double v, double w) {
    loc_status st = check_live(h);
    if (st != LOC_OK) return st;
    if (!std::isfinite(u) || !std::isfinite(v) || !std::isfinite(w))
        return fail(h, LOC_ERR_INVALID_ARG, "odometry must be finite");
    if (!odometry_advance(h, u, v, w)) return LOC_OK_DEFERRED;

    StepArgs a{};
    a.B_in = h->B[h->cur];
    a.B_out = h->B[1 - h->cur];
    a.trav = h->trav;
    a.corr = h->corr;
    a.sd = h->sd;
    a.partials = h->partials;
    a.am_pv = h->am_pv;
    a.am_pi = h->am_pi;
    a.am_idx = h->argmax_idx;
    a.am_val = h->argmax_val;
    a.inv_uniform = h->inv_uniform;
    a.out_mult = storage_mult(h->p.storage);
    a.log_out_mult = std::log((double)a.out_mult);
    a.H = h->p.H;
    a.W = h->p.W;
    a.K = h->p.K;
    a.r_xy = h->r_xy;
    a.r_th = h->r_th;
    std::memcpy(a.gx, h->gx, sizeof(a.gx));
    std::memcpy(a.gt, h->gt, sizeof(a.gt));
    shift_table(h, a.sh);
    cudaError_t e;
    if (h->aniso) {
        // channel k's heading 2 pi k / K + theta_t, theta_t reduced to [0, 2 pi) in FP64
        double th = std::fmod(h->theta, 2.0 * M_PI);
        if (th < 0.0) th += 2.0 * M_PI;
        a.phi0 = (float)th;
        a.dphi = (float)(2.0 * M_PI / a.K);
        a.sigma_a = (float)h->p.sigma_xy_cells;
        a.sigma_c = (float)h->p.sigma_cross_cells;
        e = launch_step_aniso(a, h->aniso_tma ? h->tmap[h->cur] : nullptr, h->p.storage, h->stream);
    } else {
        e = h->tiled ? launch_step_tiled(a, h->tmap[h->cur], h->p.storage, h->tile_cfg, h->stream)
                     : launch_step(a, h->p.storage, h->stream);
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "step launch");
    step_done(h);
    // the warp-specialised tiled kernels write the argmax of the new tensor
    h->am_valid = !h->aniso && h->tiled && step_tiled_fuses_argmax(h->tile_cfg);
    return LOC_OK;
}

namespace {

loc_status lidar_setup(loc_session* h) {
    if (h->lidar_ready) return LOC_OK;
    const int H = h->p.H, W = h->p.W, K = h->p.K;
    const long long hw = (long long)H * W;
    long long cap = 2LL * h->p.n_samples + 4LL * (H + W) + 1024;
    if (cap > hw) cap = hw;
    h->cap = (int)cap;
    const int nrb = (H + 31) / 32;
    h->m = (float*)dev_alloc(h, sizeof(float) * hw);
    h->travbits = (uint32_t*)dev_alloc(h, sizeof(uint32_t) * (size_t)H * ((W + 31) / 32));
    h->sel = (uint8_t*)dev_alloc(h, hw);
    h->rowcnt = (int*)dev_alloc(h, sizeof(int) * H);
    h->rowoff = (int*)dev_alloc(h, sizeof(int) * H);
    h->bnd = (float*)dev_alloc(h, sizeof(float) * (size_t)(nrb + 1) * W);
    h->prog = (int*)dev_alloc(h, sizeof(int) * (size_t)(nrb + 2));
    h->samples = (int32_t*)dev_alloc(h, sizeof(int32_t) * (size_t)cap);
    h->logL = (float*)dev_alloc(h, sizeof(float) * (size_t)cap * K);
    h->dscal = (int*)dev_alloc(h, 64);
    h->rs = dev_alloc(h, reweight_scalars_bytes());
    if (!h->m || !h->sel || !h->rowcnt || !h->rowoff || !h->bnd || !h->prog || !h->samples || !h->logL ||
        !h->dscal || !h->rs || !h->travbits)
        return fail(h, LOC_ERR_OOM, "LIDAR scratch allocation failed");
    cudaError_t e = cudaMemsetAsync(h->dscal, 0, 64, h->stream);
    if (e == cudaSuccess) e = launch_pack_bits(h->trav, H, W, h->travbits, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->rs, 0, reweight_scalars_bytes(), h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "LIDAR scratch init");
    h->lidar_ready = true;
    return LOC_OK;
}

void dev_release(loc_session* h, void* p) {
    auto it = std::find(h->owned.begin(), h->owned.end(), p);
    if (it == h->owned.end()) return;
    h->owned.erase(it);
    if (g_free) g_free(p, (void*)h->stream, g_alloc_ctx);
    else cudaFree(p);
}

// Grow a device buffer to at least n elements of `elem` bytes (the old one is released).
template <typename P>
bool grow(loc_session* h, P*& ptr, int& capn, int n, size_t elem) {
    if (n <= capn && ptr) return true;
    void* q = dev_alloc(h, elem * (size_t)std::max(n, 1));
    if (!q) return false;
    if (ptr) dev_release(h, (void*)ptr);
    ptr = (P*)q;
    capn = std::max(n, 1);
    return true;
}

// Scoring inputs for one scan: the used beams (b % stride == 0, range < r_max), their
// ranges, the distinct FP32 map-frame directions of every (bin, used beam) pair and the
// direction index of each pair.  The angle of bin k and beam b is
// (2 pi / K) k + theta_t + (angle_min + angle_inc b), evaluated in FP64 in that order; its
// cosine and sine are rounded to FP32.  Pairs with the same FP64 angle share one sincos
// (most of the K x used-beam pairs repeat an angle), and the tables go to the device through
// pinned staging, so the copies are asynchronous.
loc_status upload_scan(loc_session* h, const float* ranges, int n_beams, double angle_min, double angle_inc,
                       double r_max, int stride, int* n_used_out, int* n_dirs_out) {
    const int K = h->p.K;
    int nu = 0;
    for (int b = 0; b < n_beams; b += stride) nu += ranges[b] < r_max;
    const size_t npairs = (size_t)K * std::max(nu, 1);
    // staging slot: [dirs: 2 * npairs floats][z: nu floats][dir_of: npairs ints]
    const size_t bytes = sizeof(float) * 2 * npairs + sizeof(float) * std::max(nu, 1) + sizeof(int32_t) * npairs;
    const int slot = h->scan_slot;
    h->scan_slot ^= 1;
    if (h->scan_pin_ev[slot]) {
        cudaError_t e = cudaEventSynchronize(h->scan_pin_ev[slot]);   // its copies have run
        if (e != cudaSuccess) return cuda_fail(h, e, "scan staging");
    } else if (cudaEventCreateWithFlags(&h->scan_pin_ev[slot], cudaEventDisableTiming) != cudaSuccess) {
        h->scan_pin_ev[slot] = nullptr;
        return fail(h, LOC_ERR_OOM, "scan staging event");
    }
    if (h->scan_pin_cap[slot] < bytes) {
        if (h->scan_pin[slot]) cudaFreeHost(h->scan_pin[slot]);
        h->scan_pin[slot] = nullptr;
        h->scan_pin_cap[slot] = 0;
        const size_t want = std::max(bytes, (size_t)K * 512 * 16);       // room for 512 used beams
        void* q = nullptr;
        if (cudaMallocHost(&q, want) != cudaSuccess) {
            cudaGetLastError();
            return fail(h, LOC_ERR_OOM, "scan staging (pinned)");
        }
        h->scan_pin[slot] = static_cast<unsigned char*>(q);
        h->scan_pin_cap[slot] = want;
    }
    float* dirs = reinterpret_cast<float*>(h->scan_pin[slot]);
    float* zu = dirs + 2 * npairs;
    int32_t* dir_of = reinterpret_cast<int32_t*>(zu + std::max(nu, 1));
    std::vector<int> used;
    used.reserve((size_t)nu);
    for (int b = 0, u = 0; b < n_beams; b += stride)
        if (ranges[b] < r_max) {
            used.push_back(b);
            zu[u++] = ranges[b];
        }
    // open-addressing tables: FP64 angle bits -> (cos, sin) as FP32, and the distinct FP32
    // direction pairs (keys are the bit patterns of (cos, sin); a zero key marks an empty slot,
    // so that pattern is kept aside)
    size_t cap = 64;
    while (cap < 2 * npairs) cap <<= 1;
    std::vector<unsigned long long> akeys(cap, 0ull);
    std::vector<float> acs(2 * cap);
    std::vector<unsigned long long> keys(cap, 0ull);
    std::vector<int> ids(cap, -1);
    int zero_id = -1, nd = 0;
    const double beam0 = angle_min;
    for (int k = 0; k < K; ++k) {
        const double ak = (2.0 * M_PI / K) * k + h->theta;
        for (int u = 0; u < nu; ++u) {
            const double a = ak + (beam0 + angle_inc * used[u]);
            unsigned long long abits;
            std::memcpy(&abits, &a, 8);
            float c, sn;
            {
                const unsigned long long akey = abits ? abits : 1ull;   // 0 bits (angle +0.0): key 1, never a double's bits here otherwise
                size_t slot_a = (size_t)((akey * 0x9E3779B97F4A7C15ull) >> 40) & (cap - 1);
                while (akeys[slot_a] != 0ull && akeys[slot_a] != akey) slot_a = (slot_a + 1) & (cap - 1);
                if (akeys[slot_a] == akey) {
                    c = acs[2 * slot_a];
                    sn = acs[2 * slot_a + 1];
                } else {
                    c = (float)std::cos(a);
                    sn = (float)std::sin(a);
                    akeys[slot_a] = akey;
                    acs[2 * slot_a] = c;
                    acs[2 * slot_a + 1] = sn;
                }
            }
            unsigned int bc, bs;
            std::memcpy(&bc, &c, 4);
            std::memcpy(&bs, &sn, 4);
            const unsigned long long key = ((unsigned long long)bc << 32) | bs;
            int id = -1;
            if (key == 0ull) {
                id = zero_id;
            } else {
                size_t sl = (size_t)((key * 0x9E3779B97F4A7C15ull) >> 40) & (cap - 1);
                while (keys[sl] != 0ull && keys[sl] != key) sl = (sl + 1) & (cap - 1);
                if (keys[sl] == key) id = ids[sl];
                else keys[sl] = key;
                if (id < 0) ids[sl] = nd;
            }
            if (id < 0) {
                id = nd++;
                if (key == 0ull) zero_id = id;
                dirs[2 * id] = c;
                dirs[2 * id + 1] = sn;
            }
            dir_of[(size_t)k * nu + u] = id;
        }
    }
    // device tables sized once for this staging capacity, so steady-state scans allocate nothing
    const int cap_pairs = (int)std::min<size_t>(h->scan_pin_cap[slot] / 16, (size_t)INT_MAX / 2);
    if (!grow(h, h->dirs, h->cap_dirs, std::max(nd, cap_pairs), 2 * sizeof(float)) ||
        !grow(h, h->z, h->cap_beams, std::max(nu, cap_pairs / K), sizeof(float)) ||
        !grow(h, h->dir_of, h->cap_dir_of, std::max(K * nu, cap_pairs), sizeof(int32_t)))
        return fail(h, LOC_ERR_OOM, "scan buffers");
    cudaError_t e = cudaSuccess;
    if (nd) e = cudaMemcpyAsync(h->dirs, dirs, sizeof(float) * 2 * (size_t)nd, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess && nu)
        e = cudaMemcpyAsync(h->z, zu, sizeof(float) * nu, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess && nu)
        e = cudaMemcpyAsync(h->dir_of, dir_of, sizeof(int32_t) * (size_t)K * nu, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaEventRecord(h->scan_pin_ev[slot], h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "scan upload");
    *n_used_out = nu;
    *n_dirs_out = nd;
    return LOC_OK;
}

loc_status check_scan(loc_session* h, const float* ranges, int n_beams, double angle_min, double angle_inc,
                      double r_max, int stride, double sigma_r) {
    if (!ranges || n_beams <= 0) return fail(h, LOC_ERR_INVALID_ARG, "ranges null or n_beams <= 0");
    if (!std::isfinite(angle_min) || !std::isfinite(angle_inc) || !(r_max > 0.0) || !std::isfinite(r_max) ||
        !(sigma_r > 0.0) || !std::isfinite(sigma_r) || stride < 1)
        return fail(h, LOC_ERR_INVALID_ARG, "scan parameters: finite angles, r_max > 0, sigma_r > 0, stride >= 1");
    for (int b = 0; b < n_beams; ++b)
        if (!std::isfinite(ranges[b]) || ranges[b] < 0.0f)
            return fail(h, LOC_ERR_INVALID_ARG, "ranges must be finite and >= 0");
    return LOC_OK;
}

// Scores the sample list on the device (h->samples, count in h->dscal[0]) and reweights.
loc_status score_and_reweight(loc_session* h, int n_used, int n_dirs, double r_max, double sigma_r) {
    if (n_used == 0 || n_dirs == 0) return LOC_OK;        // nothing to score
    h->am_valid = false;
    const double cell = h->p.cell_m;
    cudaError_t e = launch_score_reweight(
        h->B[h->cur], h->p.storage, h->trav, h->travbits, h->p.H, h->p.W, h->p.K, h->samples, h->dscal, h->cap, h->dirs,
        n_dirs, h->dir_of, h->z, n_used, (float)(r_max / cell), (float)cell, (float)(1.0 / (2.0 * sigma_r * sigma_r)),
        h->logL, reinterpret_cast<unsigned int*>(h->dscal + 1), h->rs, h->partials, h->nparts, h->sd,
        h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "score/reweight launch");
    h->n_lidar += 1;
    return LOC_OK;
}

loc_status materialize(loc_session* h) {
    h->am_valid = false;
    cudaError_t e = launch_materialize(h->B[h->cur], h->p.storage, h->trav, h->sd,
                                       h->inv_uniform * storage_mult(h->p.storage), h->hw, h->p.K, h->partials,
                                       h->nparts, h->stream);
    return e == cudaSuccess ? LOC_OK : cuda_fail(h, e, "materialize");
}

}  // namespace

LOC_API loc_status loc_debug_fs_stall(int stall, double wait_limit_s) {
    if (!(wait_limit_s > 0.0) || !(wait_limit_s <= 10.0))
        return fail(nullptr, LOC_ERR_INVALID_ARG, "wait_limit_s must be in (0, 10]");
    const cudaError_t e = set_fs_wait(wait_limit_s, stall != 0);
    if (e != cudaSuccess) return fail(nullptr, LOC_ERR_CUDA, std::string("loc_debug_fs_stall: ") + cudaGetErrorString(e));
    return LOC_OK;
}

LOC_API loc_status loc_lidar_update(loc_handle h, const float* ranges, int n_beams, double angle_min,
                                    double angle_inc, double r_max, int beam_stride, double sigma_r) {
    loc_status st = check_live(h);
    if (st != LOC_OK) return st;
    st = check_scan(h, ranges, n_beams, angle_min, angle_inc, r_max, beam_stride, sigma_r);
    if (st != LOC_OK) return st;
    if ((st = lidar_setup(h)) != LOC_OK) return st;
    int nu = 0, nd = 0;
    if ((st = upload_scan(h, ranges, n_beams, angle_min, angle_inc, r_max, beam_stride, &nu, &nd)) != LOC_OK)
        return st;
    if ((st = materialize(h)) != LOC_OK) return st;
    cudaError_t e = launch_belief_map(h->B[h->cur], h->p.storage, h->trav, h->sd, h->inv_uniform, h->p.H, h->p.W,
                                      h->p.K, h->m, h->partials, h->nparts, &h->sd->counter, h->p.n_samples,
                                      reinterpret_cast<float*>(h->dscal + 2), h->stream);
    if (e == cudaSuccess)
        e = launch_dither(h->m, reinterpret_cast<float*>(h->dscal + 2), h->p.H, h->p.W, h->sel, h->rowcnt,
                          h->rowoff, h->dscal, h->bnd, h->prog, &h->sd->status, h->cap, h->samples, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "sample selection launch");
    return score_and_reweight(h, nu, nd, r_max, sigma_r);
}

LOC_API loc_status loc_lidar_update_cells(loc_handle h, const int32_t* cells, int n_cells, const float* ranges,
                                          int n_beams, double angle_min, double angle_inc, double r_max,
                                          int beam_stride, double sigma_r) {
    loc_status st = check_live(h);
    if (st != LOC_OK) return st;
    st = check_scan(h, ranges, n_beams, angle_min, angle_inc, r_max, beam_stride, sigma_r);
    if (st != LOC_OK) return st;
    if (n_cells < 0 || (n_cells > 0 && !cells) || (long long)n_cells > (long long)h->hw)
        return fail(h, LOC_ERR_INVALID_ARG, "cells null or n_cells out of range");
    std::vector<int32_t> sorted(cells, cells + n_cells);
    std::sort(sorted.begin(), sorted.end());
    for (int c = 0; c < n_cells; ++c) {
        if (sorted[c] < 0 || (size_t)sorted[c] >= h->hw) return fail(h, LOC_ERR_INVALID_ARG, "cell index out of grid");
        if (c > 0 && sorted[c] == sorted[c - 1]) return fail(h, LOC_ERR_INVALID_ARG, "duplicate cell index");
    }
    if ((st = lidar_setup(h)) != LOC_OK) return st;
    if (n_cells > h->cap) {                 // a larger sample list than dithering would give
        int32_t* s2 = (int32_t*)dev_alloc(h, sizeof(int32_t) * (size_t)n_cells);
        float* l2 = (float*)dev_alloc(h, sizeof(float) * (size_t)n_cells * h->p.K);
        if (!s2 || !l2) return fail(h, LOC_ERR_OOM, "sample buffers");
        dev_release(h, h->samples);
        dev_release(h, h->logL);
        h->samples = s2;
        h->logL = l2;
        h->cap = n_cells;
    }
    int nu = 0, nd = 0;
    if ((st = upload_scan(h, ranges, n_beams, angle_min, angle_inc, r_max, beam_stride, &nu, &nd)) != LOC_OK)
        return st;
    if ((st = materialize(h)) != LOC_OK) return st;
    cudaError_t e = cudaSuccess;
    if (n_cells)
        e = cudaMemcpyAsync(h->samples, cells, sizeof(int32_t) * n_cells, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->dscal, &n_cells, sizeof(int), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);      // n_cells lives on this stack frame
    if (e != cudaSuccess) return cuda_fail(h, e, "sample upload");
    return score_and_reweight(h, nu, nd, r_max, sigma_r);
}

LOC_API loc_status loc_samples(loc_handle h, int32_t* out, size_t cap, int* n) {
    loc_status st = check_live(h);
    if (st != LOC_OK) return st;
    if (!n || (cap > 0 && !out)) return fail(h, LOC_ERR_INVALID_ARG, "null output");
    *n = 0;
    if (!h->lidar_ready) return LOC_OK;
    int cnt = 0;
    cudaError_t e = cudaMemcpyAsync(&cnt, h->dscal, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "loc_samples");
    const int avail = std::min(cnt, h->cap);
    const size_t nout = std::min((size_t)avail, cap);
    if (nout) {
        e = cudaMemcpyAsync(out, h->samples, sizeof(int32_t) * nout, cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "loc_samples");
    }
    *n = cnt;
    return sync_and_check(h);
}

LOC_API loc_status loc_dither(loc_handle h, const float* m, float fs, uint8_t* sel, int* count) {
    loc_status st = check_live(h);
    if (st != LOC_OK) return st;
    if (!m || !sel || !count) return fail(h, LOC_ERR_INVALID_ARG, "null argument");
    if (!std::isfinite(fs)) return fail(h, LOC_ERR_INVALID_ARG, "fs must be finite");
    for (size_t q = 0; q < h->hw; ++q)
        if (!std::isfinite(m[q])) return fail(h, LOC_ERR_INVALID_ARG, "map values must be finite");
    if ((st = lidar_setup(h)) != LOC_OK) return st;
    cudaError_t e = cudaMemcpyAsync(h->m, m, sizeof(float) * h->hw, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->dscal + 2, &fs, sizeof(float), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
        e = launch_dither(h->m, reinterpret_cast<float*>(h->dscal + 2), h->p.H, h->p.W, h->sel, h->rowcnt, h->rowoff,
                          h->dscal + 3, h->bnd, h->prog, &h->sd->status, 0, nullptr, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sel, h->sel, h->hw, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(count, h->dscal + 3, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "loc_dither");
    return sync_and_check(h);
}

LOC_API loc_status loc_ray_ranges(loc_handle h, const int32_t* cells, int n_cells, const float* dirs, int n_dirs,
                                  double r_max, float* out) {
    loc_status st = check_live(h);
    if (st != LOC_OK) return st;
    if (n_cells < 0 || n_dirs < 0 || (n_cells && !cells) || (n_dirs && !dirs) || (n_cells && n_dirs && !out))
        return fail(h, LOC_ERR_INVALID_ARG, "null argument or negative count");
    if (!(r_max > 0.0) || !std::isfinite(r_max)) return fail(h, LOC_ERR_INVALID_ARG, "r_max must be > 0");
    for (int c = 0; c < n_cells; ++c)
        if (cells[c] < 0 || (size_t)cells[c] >= h->hw) return fail(h, LOC_ERR_INVALID_ARG, "cell index out of grid");
    for (int d = 0; d < 2 * n_dirs; ++d)
        if (!std::isfinite(dirs[d])) return fail(h, LOC_ERR_INVALID_ARG, "directions must be finite");
    if (!n_cells || !n_dirs) return LOC_OK;
    const size_t n = (size_t)n_cells * n_dirs;
    int32_t* dc = (int32_t*)dev_alloc(h, sizeof(int32_t) * n_cells);
    float* dd = (float*)dev_alloc(h, sizeof(float) * 2 * n_dirs);
    float* dout = (float*)dev_alloc(h, sizeof(float) * n);
    if (!dc || !dd || !dout) return fail(h, LOC_ERR_OOM, "ray buffers");
    cudaError_t e = cudaMemcpyAsync(dc, cells, sizeof(int32_t) * n_cells, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dd, dirs, sizeof(float) * 2 * n_dirs, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
        e = launch_ray_ranges(h->trav, h->p.H, h->p.W, dc, n_cells, dd, n_dirs, (float)(r_max / h->p.cell_m),
                              (float)h->p.cell_m, dout, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, dout, sizeof(float) * n, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    for (void* p : {(void*)dc, (void*)dd, (void*)dout}) dev_release(h, p);
    if (e != cudaSuccess) return cuda_fail(h, e, "loc_ray_ranges");
    return sync_and_check(h);
}

LOC_API loc_status loc_range_table(loc_handle h, int n_angles, double r_max) {
    loc_status st = check_live(h);
    if (st != LOC_OK) return st;
    if (n_angles <= 0 || n_angles > LOC_MAX_TABLE_DIRS || n_angles % h->p.K != 0)
        return fail(h, LOC_ERR_INVALID_ARG, "n_angles must be a positive multiple of K, <= LOC_MAX_TABLE_DIRS");
    if (!(r_max > 0.0) || !std::isfinite(r_max)) return fail(h, LOC_ERR_INVALID_ARG, "r_max must be finite and > 0");
    if (h->table) {
        dev_release(h, h->table);
        h->table = nullptr;
        h->table_A = 0;
    }
    uint8_t* t = (uint8_t*)dev_alloc(h, (size_t)n_angles * h->hw);
    float* dd = (float*)dev_alloc(h, sizeof(float) * 2 * (size_t)n_angles);
    if (!t || !dd) return fail(h, LOC_ERR_OOM, "range table");
    // table direction a: 2 pi a / A, its unit vector in FP64 rounded to FP32
    std::vector<float> dirs(2 * (size_t)n_angles);
    for (int a = 0; a < n_angles; ++a) {
        const double ang = (2.0 * M_PI / n_angles) * a;
        dirs[2 * a] = (float)std::cos(ang);
        dirs[2 * a + 1] = (float)std::sin(ang);
    }
    const float rmax_cells = (float)(r_max / h->p.cell_m);
    const float inv_step = (float)(255.0 / (double)rmax_cells);
    cudaError_t e = cudaMemcpyAsync(dd, dirs.data(), sizeof(float) * dirs.size(), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = launch_range_table(h->trav, h->p.H, h->p.W, dd, n_angles, rmax_cells, inv_step, t, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    dev_release(h, dd);
    if (e != cudaSuccess) return cuda_fail(h, e, "loc_range_table");
    h->table = t;
    h->table_A = n_angles;
    h->table_rmax = r_max;
    return sync_and_check(h);
}

LOC_API loc_status loc_range_table_read(loc_handle h, uint8_t* out, size_t n) {
    loc_status st = check_live(h);
    if (st != LOC_OK) return st;
    if (!h->table) return fail(h, LOC_ERR_INVALID_ARG, "no range table: call loc_range_table first");
    if (!out || n != (size_t)h->table_A * h->hw) return fail(h, LOC_ERR_INVALID_ARG, "out null or n != n_angles*H*W");
    cudaError_t e = cudaMemcpyAsync(out, h->table, n, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "loc_range_table_read");
    return sync_and_check(h);
}

LOC_API loc_status loc_lidar_update_dense(loc_handle h, const float* ranges, int n_beams, double angle_min,
                                          double angle_inc, int beam_stride, double sigma_r) {
    loc_status st = check_live(h);
    if (st != LOC_OK) return st;
    if (!h->table) return fail(h, LOC_ERR_INVALID_ARG, "no range table: call loc_range_table first");
    const double r_max = h->table_rmax;
    st = check_scan(h, ranges, n_beams, angle_min, angle_inc, r_max, beam_stride, sigma_r);
    if (st != LOC_OK) return st;
    const int A = h->table_A, K = h->p.K;
    // the used beams: offsets from the bin heading rounded to the table grid, ranges in code steps
    const double step = (double)(float)(r_max / 255.0);
    std::vector<int> mb;
    std::vector<float> zs;
    for (int b = 0; b < n_beams; b += beam_stride) {
        if (!(ranges[b] < r_max)) continue;
        const double x = (h->theta + (angle_min + angle_inc * b)) / (2.0 * M_PI / A);
        long long q = (long long)std::floor(x + 0.5) % A;
        if (q < 0) q += A;
        mb.push_back((int)q);
        zs.push_back((float)((double)ranges[b] / step));
    }
    const int nu = (int)mb.size();
    if (nu > LOC_MAX_DENSE_BEAMS) return fail(h, LOC_ERR_INVALID_ARG, "more than LOC_MAX_DENSE_BEAMS used beams");
    if (nu == 0) return LOC_OK;                       // every beam a dropout: nothing to weigh
    if (!h->dense_logL) {
        h->dense_logL = (float*)dev_alloc(h, sizeof(float) * h->n);
        h->dense_max = (unsigned int*)dev_alloc(h, 16);
        if (!h->dense_logL || !h->dense_max) return fail(h, LOC_ERR_OOM, "dense scan buffers");
    }
    if (!grow(h, h->dense_m, h->cap_dense, nu, sizeof(int)) || !grow(h, h->dense_z, h->cap_dense_z, nu, sizeof(float)))
        return fail(h, LOC_ERR_OOM, "dense scan buffers");
    if ((st = materialize(h)) != LOC_OK) return st;
    cudaError_t e = cudaMemcpyAsync(h->dense_m, mb.data(), sizeof(int) * nu, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->dense_z, zs.data(), sizeof(float) * nu, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->dense_max, 0, sizeof(unsigned int), h->stream);
    if (e == cudaSuccess)
        e = launch_dense_score(h->table, h->trav, h->B[h->cur], h->p.storage, h->p.H, h->p.W, K, A, h->dense_m,
                               h->dense_z, nu, (float)(step * step / (2.0 * sigma_r * sigma_r)), h->dense_logL,
                               h->dense_max, h->stream);
    h->am_valid = false;
    if (e == cudaSuccess)
        e = launch_dense_apply(h->B[h->cur], h->p.storage, h->dense_logL, (size_t)h->p.H * h->p.W, K, h->dense_max,
                               (float)std::log((double)storage_mult(h->p.storage)), h->partials, h->nparts, h->sd,
                               h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "dense scan update launch");
    h->n_dense += 1;
    return LOC_OK;
}

LOC_API loc_status loc_map_difficulty(loc_handle h, const int32_t* probes, int n_probes, int probe_bin,
                                      int beam_step, double sigma_r, double c_m, double* errors, int* n_wrong) {
    loc_status st = check_live(h);
    if (st != LOC_OK) return st;
    if (!h->table) return fail(h, LOC_ERR_INVALID_ARG, "no range table: call loc_range_table first");
    if (!probes || n_probes <= 0 || !n_wrong) return fail(h, LOC_ERR_INVALID_ARG, "null argument or n_probes <= 0");
    const int A = h->table_A, K = h->p.K, s = A / K;
    if (probe_bin < 0 || probe_bin >= K || beam_step < 1 || !(sigma_r > 0.0) || !std::isfinite(sigma_r) ||
        !(c_m >= 0.0) || !std::isfinite(c_m))
        return fail(h, LOC_ERR_INVALID_ARG, "probe_bin in [0, K), beam_step >= 1, sigma_r > 0, c_m >= 0");
    if ((A + beam_step - 1) / beam_step > LOC_MAX_DENSE_BEAMS)
        return fail(h, LOC_ERR_INVALID_ARG, "more than LOC_MAX_DENSE_BEAMS probe beams");
    for (int p = 0; p < n_probes; ++p)
        if (probes[p] < 0 || (size_t)probes[p] >= h->hw) return fail(h, LOC_ERR_INVALID_ARG, "probe out of grid");
    // the probes' table columns and map flags
    int32_t* dp = (int32_t*)dev_alloc(h, sizeof(int32_t) * n_probes);
    uint8_t* dcol = (uint8_t*)dev_alloc(h, (size_t)n_probes * A);
    uint8_t* dflag = (uint8_t*)dev_alloc(h, (size_t)n_probes);
    long long* didx = (long long*)dev_alloc(h, sizeof(long long) * n_probes);
    void* scratch = dev_alloc(h, argmax_f32_scratch_bytes());
    auto release = [&]() { for (void* q : {(void*)dp, (void*)dcol, (void*)dflag, (void*)didx, scratch}) dev_release(h, q); };
    if (!dp || !dcol || !dflag || !didx || !scratch) {
        release();
        return fail(h, LOC_ERR_OOM, "map difficulty buffers");
    }
    std::vector<uint8_t> col((size_t)n_probes * A), flag(n_probes);
    cudaError_t e = cudaMemcpyAsync(dp, probes, sizeof(int32_t) * n_probes, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(scratch, 0, argmax_f32_scratch_bytes(), h->stream);
    if (e == cudaSuccess) e = launch_gather_columns(h->table, h->trav, h->p.H, h->p.W, A, dp, n_probes, dcol, dflag, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(col.data(), dcol, col.size(), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(flag.data(), dflag, flag.size(), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        release();
        return cuda_fail(h, e, "loc_map_difficulty gather");
    }
    for (int p = 0; p < n_probes; ++p)
        if (!flag[p]) {
            release();
            return fail(h, LOC_ERR_INVALID_ARG, "probe on an occupied cell");
        }
    // each probe's noise-free scan: beams on table directions probe_bin s + b beam_step, the
    // code as the range in code steps; code 255 (capped) skipped
    std::vector<int> mall;
    std::vector<float> zall;
    std::vector<int> off(n_probes + 1, 0);
    for (int p = 0; p < n_probes; ++p) {
        for (int o = 0; o < A; o += beam_step) {
            const uint8_t code = col[(size_t)p * A + (probe_bin * s + o) % A];
            if (code == 255) continue;
            mall.push_back(o);
            zall.push_back((float)code);
        }
        off[p + 1] = (int)mall.size();
    }
    int* dm = (int*)dev_alloc(h, sizeof(int) * std::max<size_t>(mall.size(), 1));
    float* dz = (float*)dev_alloc(h, sizeof(float) * std::max<size_t>(zall.size(), 1));
    if (!h->dense_logL) {
        h->dense_logL = (float*)dev_alloc(h, sizeof(float) * h->n);
        h->dense_max = (unsigned int*)dev_alloc(h, 16);
    }
    if (!dm || !dz || !h->dense_logL || !h->dense_max) {
        release();
        if (dm) dev_release(h, dm);
        if (dz) dev_release(h, dz);
        return fail(h, LOC_ERR_OOM, "map difficulty buffers");
    }
    if (!mall.empty()) {
        e = cudaMemcpyAsync(dm, mall.data(), sizeof(int) * mall.size(), cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dz, zall.data(), sizeof(float) * zall.size(), cudaMemcpyHostToDevice, h->stream);
    }
    const double step = (double)(float)(h->table_rmax / 255.0);
    const float scale = (float)(step * step / (2.0 * sigma_r * sigma_r));
    for (int p = 0; p < n_probes && e == cudaSuccess; ++p) {
        const int nu = off[p + 1] - off[p];           // 0: every free state scores 0
        e = launch_dense_score(h->table, h->trav, h->B[h->cur], h->p.storage, h->p.H, h->p.W, K, A, dm + off[p],
                               dz + off[p], nu, scale, h->dense_logL, h->dense_max, h->stream);
        if (e == cudaSuccess) e = launch_argmax_f32(h->dense_logL, h->n, scratch, didx + p, h->stream);
    }
    std::vector<long long> idx(n_probes);
    if (e == cudaSuccess) e = cudaMemcpyAsync(idx.data(), didx, sizeof(long long) * n_probes, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    release();
    dev_release(h, dm);
    dev_release(h, dz);
    if (e != cudaSuccess) return cuda_fail(h, e, "loc_map_difficulty");
    int wrong = 0;
    const long long hw = (long long)h->hw, W = h->p.W;
    for (int p = 0; p < n_probes; ++p) {
        const long long rem = idx[p] % hw;
        const double dj = (double)(rem / W - probes[p] / W), di = (double)(rem % W - probes[p] % W);
        const double ep = h->p.cell_m * std::hypot(dj, di);
        if (errors) errors[p] = ep;
        wrong += ep > c_m;
    }
    *n_wrong = wrong;
    return sync_and_check(h);
}

LOC_API loc_status loc_belief(loc_handle h, float* out, size_t n) {
    loc_status st = check_live(h);
    if (st != LOC_OK) return st;
    if (!out || n != h->n) return fail(h, LOC_ERR_INVALID_ARG, "out null or n != K*H*W");
    float* tmp = (float*)dev_alloc(h, n * sizeof(float));
    if (!tmp) return fail(h, LOC_ERR_OOM, "readback buffer");
    cudaError_t e = launch_read_belief(h->B[h->cur], h->p.storage, h->trav, h->sd, h->inv_uniform,
                                       h->p.H, h->p.W, h->p.K, tmp, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, tmp, n * sizeof(float), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    h->owned.pop_back();
    if (g_free) g_free(tmp, (void*)h->stream, g_alloc_ctx); else cudaFree(tmp);
    if (e != cudaSuccess) return cuda_fail(h, e, "loc_belief");
    return sync_and_check(h);
}

LOC_API loc_status loc_marginal(loc_handle h, float* out, size_t n, int mode) {
    loc_status st = check_live(h);
    if (st != LOC_OK) return st;
    if (!out || n != h->hw) return fail(h, LOC_ERR_INVALID_ARG, "out null or n != H*W");
    if (mode != LOC_MAP_SUM && mode != LOC_MAP_MAX) return fail(h, LOC_ERR_INVALID_ARG, "mode");
    float* tmp = (float*)dev_alloc(h, n * sizeof(float));
    if (!tmp) return fail(h, LOC_ERR_OOM, "readback buffer");
    cudaError_t e = launch_read_marginal(h->B[h->cur], h->p.storage, h->trav, h->sd, h->inv_uniform,
                                         h->p.H, h->p.W, h->p.K, mode, tmp, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, tmp, n * sizeof(float), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    h->owned.pop_back();
    if (g_free) g_free(tmp, (void*)h->stream, g_alloc_ctx); else cudaFree(tmp);
    if (e != cudaSuccess) return cuda_fail(h, e, "loc_marginal");
    return sync_and_check(h);
}

LOC_API loc_status loc_argmax(loc_handle h, int* k, int* j, int* i, float* p) {
    loc_status st = check_live(h);
    if (st != LOC_OK) return st;
    if (!k || !j || !i || !p) return fail(h, LOC_ERR_INVALID_ARG, "null output");
    long long idx = -1;
    float val = 0.0f;
    int status = 0;
    // after a tiled propagation the step itself left the argmax of the new tensor (or -1 when
    // it restarted); otherwise, or then, one pass over the stored tensor
    for (int pass = h->am_valid ? 0 : 1; pass < 2 && idx < 0; ++pass) {
        cudaError_t e = cudaSuccess;
        if (pass == 1)
            e = launch_argmax(h->B[h->cur], h->p.storage, h->trav, h->sd, h->inv_uniform, h->p.H, h->p.W, h->p.K,
                              h->argmax_scratch, h->argmax_idx, h->argmax_val, h->stream);
        // the result and the device status in one round trip, through pinned memory
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h->pinned, h->argmax_idx, sizeof(long long) + sizeof(float),
                                cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h->pinned + 16, &h->sd->status, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "loc_argmax");
        std::memcpy(&idx, h->pinned, sizeof(idx));
        std::memcpy(&val, h->pinned + sizeof(long long), sizeof(val));
        std::memcpy(&status, h->pinned + 16, sizeof(status));
        if (status != 0) break;
    }
    const loc_status cs = check_status(h, status);
    if (cs != LOC_OK) return cs;
    if (idx < 0) return fail(h, LOC_ERR_CUDA, "loc_argmax: no result");
    h->am_valid = true;                    // the buffer holds the argmax of the current tensor
    const long long hw = (long long)h->hw;
    *k = (int)(idx / hw);
    *j = (int)((idx % hw) / h->p.W);
    *i = (int)(idx % h->p.W);
    *p = val;
    return check_status(h, status);
}

LOC_API loc_status loc_estimate(loc_handle h, double radius_m, int dk, loc_estimate_t* out) {
    loc_status st = check_live(h);
    if (st != LOC_OK) return st;
    if (!out) return fail(h, LOC_ERR_INVALID_ARG, "null output");
    if (!(radius_m >= 0.0) || !std::isfinite(radius_m) || dk < 0)
        return fail(h, LOC_ERR_INVALID_ARG, "radius_m must be finite and >= 0, dk >= 0");
    if (!h->est) {
        h->est = (EstimateOut*)dev_alloc(h, sizeof(EstimateOut));
        if (!h->est) return fail(h, LOC_ERR_OOM, "estimate buffer");
    }
    const double c = h->p.cell_m;
    // cells whose centres lie within radius_m; the 1e-9 keeps a whole number of cells inclusive
    const double r2d = std::floor(radius_m * radius_m / (c * c) + 1e-9);
    const long long r2 = r2d > 4.0e18 ? (long long)4e18 : (long long)r2d;
    cudaError_t e = launch_argmax(h->B[h->cur], h->p.storage, h->trav, h->sd, h->inv_uniform, h->p.H, h->p.W, h->p.K,
                                  h->argmax_scratch, h->argmax_idx, h->argmax_val, h->stream);
    if (e == cudaSuccess)
        e = launch_estimate(h->B[h->cur], h->p.storage, h->trav, h->sd, h->inv_uniform, h->p.H, h->p.W, h->p.K,
                            h->argmax_scratch, h->argmax_idx, r2, dk, h->partials, h->nparts, h->est, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->pinned, h->argmax_idx, sizeof(long long) + sizeof(float), cudaMemcpyDeviceToHost,
                            h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->pinned + 16, &h->sd->status, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->pinned + 24, h->est, sizeof(EstimateOut), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "loc_estimate");
    long long idx;
    float val;
    int status;
    EstimateOut eo;
    std::memcpy(&idx, h->pinned, sizeof(idx));
    std::memcpy(&val, h->pinned + sizeof(long long), sizeof(val));
    std::memcpy(&status, h->pinned + 16, sizeof(status));
    std::memcpy(&eo, h->pinned + 24, sizeof(eo));
    const long long hw = (long long)h->hw;
    out->k = (int)(idx / hw);
    out->j = (int)((idx % hw) / h->p.W);
    out->i = (int)(idx % h->p.W);
    out->x = (out->i + 0.5) * c;
    out->y = (out->j + 0.5) * c;
    double th = std::fmod(2.0 * M_PI * out->k / h->p.K + h->theta, 2.0 * M_PI);
    if (th < 0.0) th += 2.0 * M_PI;
    out->theta = th;
    out->p = val;
    out->mass_near = eo.mass_near;
    out->second_j = eo.second_cell >= 0 ? (int)(eo.second_cell / h->p.W) : -1;
    out->second_i = eo.second_cell >= 0 ? (int)(eo.second_cell % h->p.W) : -1;
    out->second_p = eo.second_p;
    out->second_ratio = val > 0.0f ? (double)eo.second_p / (double)val : 0.0;
    return check_status(h, status);
}

LOC_API loc_status loc_set_belief(loc_handle h, const float* b, size_t n) {
    loc_status st = check_live(h);
    if (st != LOC_OK) return st;
    if (!b || n != h->n) return fail(h, LOC_ERR_INVALID_ARG, "b null or n != K*H*W");
    double sum = 0.0;
    for (size_t q = 0; q < n; ++q) {
        if (!std::isfinite(b[q]) || b[q] < 0.0f)
            return fail(h, LOC_ERR_INVALID_ARG, "belief values must be finite and >= 0");
        sum += b[q];
    }
    if (!(sum > 0.0)) return fail(h, LOC_ERR_INVALID_ARG, "belief sums to 0");
    float* tmp = (float*)dev_alloc(h, n * sizeof(float));
    if (!tmp) return fail(h, LOC_ERR_OOM, "upload buffer");
    h->am_valid = false;
    cudaError_t e = cudaMemcpyAsync(tmp, b, n * sizeof(float), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
        e = launch_set_belief(tmp, h->B[h->cur], h->p.storage, n, h->sd, h->partials, h->nparts, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    h->owned.pop_back();
    if (g_free) g_free(tmp, (void*)h->stream, g_alloc_ctx); else cudaFree(tmp);
    if (e != cudaSuccess) return cuda_fail(h, e, "loc_set_belief");
    return sync_and_check(h);
}

LOC_API loc_status loc_stats(loc_handle h, double* theta_t, double* last_Z, double* logscale,
                             long long* n_propagations, long long* n_reinit) {
    loc_status st = check_live(h);
    if (st != LOC_OK) return st;
    SessionDev d{};
    cudaError_t e = cudaMemcpyAsync(&d, h->sd, sizeof(d), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "loc_stats");
    if (theta_t) *theta_t = h->theta;
    if (last_Z) *last_Z = d.reinit && d.n_reinit ? 0.0 : d.Z / (double)storage_mult(h->p.storage);
    if (logscale) *logscale = d.logscale;
    if (n_propagations) *n_propagations = h->n_prop;
    if (n_reinit) *n_reinit = (long long)d.n_reinit;
    return sync_and_check(h);
}

LOC_API loc_status loc_sync(loc_handle h) {
    loc_status st = check_live(h);
    if (st != LOC_OK) return st;
    return sync_and_check(h);
}

LOC_API loc_status loc_destroy(loc_handle h) {
    if (!h) return LOC_OK;
    cudaStreamSynchronize(h->stream);
    release_all(h);
    delete h;
    return LOC_OK;
}

LOC_API const char* loc_last_error(loc_handle h) {
    return h ? h->err.c_str() : g_thread_err.c_str();
}
