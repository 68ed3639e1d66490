// C-ABI of the localizer: session state on the host, device buffers, odometry bookkeeping
// (Section III-A, Eq. 2, the Alg. 1 gate) and the launches of the device kernels.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "kernels.h"

#define LOC_API extern "C" __attribute__((visibility("default")))

using namespace loc;

namespace {

thread_local std::string g_thread_err;
loc_alloc_fn g_alloc = nullptr;
loc_free_fn g_free = nullptr;
void* g_alloc_ctx = nullptr;

}  // namespace

void loc::set_thread_error(const char* msg) { g_thread_err = msg ? msg : ""; }

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
    SessionDev* sd = nullptr;
    double* partials = nullptr;
    unsigned int nparts = 0;
    void* argmax_scratch = nullptr;
    long long* argmax_idx = nullptr;
    float* argmax_val = nullptr;
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

namespace {

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

int radius(double sigma, int given) {
    if (given >= 0) return given;
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
    int status = 0;
    e = cudaMemcpy(&status, &h->sd->status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemcpy(status)");
    if (status & LOC_DEV_ERR_TIMEOUT) return fail(h, LOC_ERR_TIMEOUT, "device wait timed out");
    if (status & LOC_DEV_ERR_NONFINITE_Z) {
        h->failed = true;
        return fail(h, LOC_ERR_STATE, "normaliser was not finite");
    }
    return LOC_OK;
}

}  // namespace

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
}

LOC_API void loc_set_allocator(loc_alloc_fn alloc, loc_free_fn release, void* ctx) {
    g_alloc = (alloc && release) ? alloc : nullptr;
    g_free = (alloc && release) ? release : nullptr;
    g_alloc_ctx = (alloc && release) ? ctx : nullptr;
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
    const int rxy = radius(p->sigma_xy_cells, p->r_xy), rth = radius(p->sigma_theta_bins, p->r_theta);
    if (rxy > LOC_MAX_R_XY || rth > LOC_MAX_R_THETA)
        return fail(nullptr, LOC_ERR_INVALID_ARG, "kernel radius above LOC_MAX_R_XY / LOC_MAX_R_THETA");
    if (p->n_samples < 0) return fail(nullptr, LOC_ERR_INVALID_ARG, "n_samples must be >= 0");
    if (p->kernel < LOC_KERNEL_AUTO || p->kernel > LOC_KERNEL_TILED)
        return fail(nullptr, LOC_ERR_INVALID_ARG, "unknown kernel selection");
    const bool tiled_ok = step_tiled_eligible(p->H, p->W, p->K, rxy, rth, p->storage);
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
    s->argmax_scratch = dev_alloc(s, argmax_scratch_bytes(s->n));
    s->argmax_idx = (long long*)dev_alloc(s, sizeof(long long) + sizeof(float));
    if (!s->B[0] || !s->B[1] || !s->trav || !s->corr || !s->sd || !s->partials ||
        !s->argmax_scratch || !s->argmax_idx) {
        release_all(s);
        delete s;
        return fail(nullptr, LOC_ERR_OOM, "device allocation failed");
    }
    s->argmax_val = (float*)(s->argmax_idx + 1);
    s->tiled = tiled_ok && p->kernel != LOC_KERNEL_GENERIC;
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

LOC_API loc_status loc_step(loc_handle h, double u, double v, double w) {
    loc_status st = check_live(h);
    if (st != LOC_OK) return st;
    if (!std::isfinite(u) || !std::isfinite(v) || !std::isfinite(w))
        return fail(h, LOC_ERR_INVALID_ARG, "odometry must be finite");
    // Section III-A / Eq. 2: translate in the frame of theta_{t-1}, then rotate.
    const double c = std::cos(h->theta), s = std::sin(h->theta);
    h->px += c * u - s * v;
    h->py += s * u + c * v;
    h->theta += w;
    const double cell = h->p.cell_m;
    if (std::hypot(h->px, h->py) / cell < h->p.min_shift_cells) return LOC_OK_DEFERRED;

    StepArgs a{};
    a.B_in = h->B[h->cur];
    a.B_out = h->B[1 - h->cur];
    a.trav = h->trav;
    a.corr = h->corr;
    a.sd = h->sd;
    a.partials = h->partials;
    a.inv_uniform = h->inv_uniform;
    a.out_mult = storage_mult(h->p.storage);
    a.log_out_mult = std::log((double)a.out_mult);
    a.seed = pcg_hash((uint32_t)h->n_prop * 0x9E3779B9u + 0x632BE5ABu);
    a.H = h->p.H;
    a.W = h->p.W;
    a.K = h->p.K;
    a.r_xy = h->r_xy;
    a.r_th = h->r_th;
    std::memcpy(a.gx, h->gx, sizeof(a.gx));
    std::memcpy(a.gt, h->gt, sizeof(a.gt));
    const int K = h->p.K;
    for (int k = 0; k < K; ++k) {
        const double ang = 2.0 * M_PI * k / K;
        const double ck = std::cos(ang), sk = std::sin(ang);
        const double sx = (ck * h->px - sk * h->py) / cell;   // Eq. 2: R(k dTheta) p, in cells
        const double sy = (sk * h->px + ck * h->py) / cell;
        // Eq. 3 pull source: integer part and fraction of -s.  A fraction within 1e-9 of a
        // whole cell (e.g. 3 cos(pi/2) = 1.8e-16) is snapped, which changes the result by
        // under 1e-9 relative and keeps integer shifts exact permutations.
        double ox = std::floor(-sx), oy = std::floor(-sy);
        double fx = -sx - ox, fy = -sy - oy;
        if (fx < 1e-9) fx = 0.0;
        if (fx > 1.0 - 1e-9) { fx = 0.0; ox += 1.0; }
        if (fy < 1e-9) fy = 0.0;
        if (fy > 1.0 - 1e-9) { fy = 0.0; oy += 1.0; }
        a.sh[k].ox = (int)ox;
        a.sh[k].oy = (int)oy;
        a.sh[k].fx = (float)fx;
        a.sh[k].fy = (float)fy;
    }
    cudaError_t e = h->tiled ? launch_step_tiled(a, h->tmap[h->cur], h->p.storage, h->tile_cfg, h->stream)
                             : launch_step(a, h->p.storage, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "step launch");
    h->cur = 1 - h->cur;
    h->px = h->py = 0.0;
    h->n_prop += 1;
    return LOC_OK;
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
    cudaError_t e = launch_argmax(h->B[h->cur], h->p.storage, h->trav, h->sd, h->inv_uniform,
                                  h->p.H, h->p.W, h->p.K, h->argmax_scratch, h->argmax_idx,
                                  h->argmax_val, h->stream);
    struct { long long idx; float val; } res{};
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&res, h->argmax_idx, sizeof(long long) + sizeof(float),
                            cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "loc_argmax");
    const long long hw = (long long)h->hw;
    *k = (int)(res.idx / hw);
    *j = (int)((res.idx % hw) / h->p.W);
    *i = (int)(res.idx % h->p.W);
    *p = res.val;
    return sync_and_check(h);
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
