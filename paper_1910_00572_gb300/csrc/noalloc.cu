// Allocation-free propagation entry point.
//
// Some callers cannot allocate device memory at the time they propagate: code running under
// a strict real-time budget where a cudaMalloc could stall, embedded or safety-certified
// stacks whose memory is reserved once at start-up, and hosts whose allocator is owned by
// another runtime.  loc_propagate_noalloc serves them: the caller passes its own device
// buffers for the inputs and outputs, and the only other memory the kernel touches is a
// fixed scratch array compiled into this library (below), which every GPU that loads the
// library keeps until the process exits.
//
// The kernel is an FP32 variant of the generic propagation kernel: the same per-channel
// bilinear shift, map mask, separable Gaussian blur and circular theta blur, but the edge
// correction G(M)^-1 is recomputed per tile from the map (no precomputed field), the input
// is used as given (no session normaliser), and the FP64 block partials and the arrival
// counter live in the static scratch array.
#include <cmath>
#include <cstdio>
#include <mutex>

#include "kernels.h"

#define LOC_API extern "C" __attribute__((visibility("default")))

namespace loc {
namespace {

constexpr int TH = kGenTH, TW = kGenTW, NT = 256;
constexpr int RM = LOC_MAX_R_XY, RTM = LOC_MAX_R_THETA;
constexpr int RAW_H = TH + 2 * RM + 1, RAW_W = TW + 2 * RM + 1;
constexpr int S_H = TH + 2 * RM, S_W = TW + 2 * RM;
constexpr int RING = 2 * RTM + 1;

// Scratch shared by every call on a device: the arrival counter and one FP64 partial sum
// per CTA.  kNoAllocMaxBlocks CTAs of 16 x 32 cells cover grids up to 8192 tiles, e.g.
// 2048 x 2048 cells.  64 KiB + 256 B.
constexpr unsigned int kNoAllocMaxBlocks = 8192;
struct NoAllocScratch {
    unsigned int counter;
    unsigned int pad[63];
    double partials[kNoAllocMaxBlocks];
};
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

struct NoAllocArgs {
    const float* B_in;
    float* B_out;
    const uint8_t* occ;            // nonzero = occupied
    double* z_out;
    NoAllocScratch* scratch;       // device address of g_noalloc_scratch
    int H, W, K;
    int r_xy, r_th;
    float gx[2 * LOC_MAX_R_XY + 1];
    float gt[2 * LOC_MAX_R_THETA + 1];
    Shift sh[LOC_MAX_K];
};

__global__ void __launch_bounds__(NT) propagate_noalloc_kernel(const __grid_constant__ NoAllocArgs a) {
    __shared__ float raw[RAW_H][RAW_W + 1];
    __shared__ float S[S_H][S_W + 1];
    __shared__ float Xb[S_H][TW + 1];
    __shared__ float P[RING][TH][TW + 1];
    __shared__ float Mt[S_H][S_W + 1];
    __shared__ float Ct[TH][TW + 1];
    __shared__ double red[NT / 32];

    const int tid = threadIdx.x;
    const int H = a.H, W = a.W, K = a.K, r = a.r_xy, rt = a.r_th;
    const int ty0 = blockIdx.y * TH, tx0 = blockIdx.x * TW;
    const int sh_h = TH + 2 * r, sh_w = TW + 2 * r;
    const int rw_h = sh_h + 1, rw_w = sh_w + 1;
    const int ring = 2 * rt + 1;

    for (int q = tid; q < sh_h * sh_w; q += NT) {
        const int jj = q / sh_w, ii = q % sh_w;
        const int j = ty0 - r + jj, i = tx0 - r + ii;
        Mt[jj][ii] = (j >= 0 && j < H && i >= 0 && i < W && a.occ[(size_t)j * W + i] == 0) ? 1.0f : 0.0f;
    }
    __syncthreads();
    // Eq. 8 per tile: G(M) = x/y blur of M (rows first, then columns); corr = M / G(M)
    for (int q = tid; q < TH * TW; q += NT) {
        const int j = q / TW, i = q % TW;
        float G = 0.0f;
        for (int dj = -r; dj <= r; ++dj) {
            float row = 0.0f;
            for (int di = -r; di <= r; ++di) row += a.gx[di + r] * Mt[j + r + dj][i + r + di];
            G += a.gx[dj + r] * row;
        }
        Ct[j][i] = (Mt[j + r][i + r] > 0.0f && G > 0.0f) ? 1.0f / G : 0.0f;
    }

    double acc = 0.0;
    for (int kk = -rt; kk < K + rt; ++kk) {
        const int c = ((kk % K) + K) % K;
        const Shift s = a.sh[c];
        const float* plane = a.B_in + (size_t)c * H * W;
        for (int q = tid; q < rw_h * rw_w; q += NT) {
            const int jj = q / rw_w, ii = q % rw_w;
            const int j = ty0 - r + s.oy + jj, i = tx0 - r + s.ox + ii;
            raw[jj][ii] = (j >= 0 && j < H && i >= 0 && i < W) ? plane[(size_t)j * W + i] : 0.0f;
        }
        __syncthreads();
        const float fx = s.fx, fy = s.fy, gx0 = 1.0f - fx, gy0 = 1.0f - fy;
        for (int q = tid; q < sh_h * sh_w; q += NT) {
            const int jj = q / sh_w, ii = q % sh_w;
            const float top = gx0 * raw[jj][ii] + fx * raw[jj][ii + 1];
            const float bot = gx0 * raw[jj + 1][ii] + fx * raw[jj + 1][ii + 1];
            S[jj][ii] = Mt[jj][ii] * (gy0 * top + fy * bot);
        }
        __syncthreads();
        for (int q = tid; q < sh_h * TW; q += NT) {
            const int jj = q / TW, i = q % TW;
            float v = 0.0f;
            for (int d = -r; d <= r; ++d) v += a.gx[d + r] * S[jj][i + r + d];
            Xb[jj][i] = v;
        }
        __syncthreads();
        const int slot = (kk + rt) % ring;
        for (int q = tid; q < TH * TW; q += NT) {
            const int j = q / TW, i = q % TW;
            float v = 0.0f;
            for (int d = -r; d <= r; ++d) v += a.gx[d + r] * Xb[j + r + d][i];
            P[slot][j][i] = v;
        }
        __syncthreads();
        if (kk >= rt) {
            const int o = kk - rt;
            float* oplane = a.B_out + (size_t)o * H * W;
            float part = 0.0f;
            for (int q = tid; q < TH * TW; q += NT) {
                const int j = q / TW, i = q % TW;
                const int gj = ty0 + j, gi = tx0 + i;
                if (gj >= H || gi >= W) continue;
                float v = 0.0f;
                for (int d = -rt; d <= rt; ++d) v += a.gt[d + rt] * P[(o + d + rt) % ring][j][i];
                v = Ct[j][i] * v;
                oplane[(size_t)gj * W + gi] = v;
                part += v;
            }
            acc += (double)part;
        }
        __syncthreads();
    }

    const double bt = block_sum<NT>(acc, red);
    double* z_out = a.z_out;
    finish_sum<NT>(bt, a.scratch->partials, &a.scratch->counter, gridDim.x * gridDim.y, red,
                   [z_out](double Z) { *z_out = Z; });
}

// Device address of g_noalloc_scratch per device, resolved once with that device current.
std::mutex g_setup_mu;
NoAllocScratch* g_scratch_addr[128] = {};

cudaError_t scratch_for_current_device(NoAllocScratch** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = static_cast<NoAllocScratch*>(p);
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

loc_status noalloc_fail(loc_status s, const char* msg) {
    set_thread_error(msg);
    return s;
}

}  // namespace
}  // namespace loc

LOC_API loc_status loc_propagate_noalloc(const loc_params* p, const uint8_t* occ_dev,
                                         const float* b_in_dev, float* b_out_dev,
                                         double* z_out_dev, double dx_m, double dy_m) {
    using namespace loc;
    if (!p || !occ_dev || !b_in_dev || !b_out_dev || !z_out_dev)
        return noalloc_fail(LOC_ERR_INVALID_ARG, "null argument");
    if (p->H <= 0 || p->W <= 0 || p->K <= 0 || p->K > LOC_MAX_K)
        return noalloc_fail(LOC_ERR_INVALID_ARG, "H, W must be > 0 and 0 < K <= LOC_MAX_K");
    if (p->storage != LOC_F32) return noalloc_fail(LOC_ERR_INVALID_ARG, "storage must be LOC_F32");
    if (!(p->cell_m > 0.0) || !std::isfinite(p->cell_m) || !std::isfinite(dx_m) || !std::isfinite(dy_m))
        return noalloc_fail(LOC_ERR_INVALID_ARG, "cell_m and the translation must be finite, cell_m > 0");
    if (!(p->sigma_xy_cells >= 0.0) || !(p->sigma_theta_bins >= 0.0) || !std::isfinite(p->sigma_xy_cells) ||
        !std::isfinite(p->sigma_theta_bins) || !std::isfinite(p->sigma_cross_cells))
        return noalloc_fail(LOC_ERR_INVALID_ARG, "sigmas must be finite and >= 0");
    if (p->sigma_cross_cells != 0.0 && p->sigma_cross_cells != p->sigma_xy_cells)
        return noalloc_fail(LOC_ERR_INVALID_ARG, "anisotropic noise (sigma_cross_cells) needs a session (loc_create)");
    // the default radius ceil(3 sigma) is checked against the maxima before any conversion to int
    if ((p->r_xy < 0 && 3.0 * p->sigma_xy_cells > LOC_MAX_R_XY) ||
        (p->r_theta < 0 && 3.0 * p->sigma_theta_bins > LOC_MAX_R_THETA))
        return noalloc_fail(LOC_ERR_INVALID_ARG, "kernel radius above LOC_MAX_R_XY / LOC_MAX_R_THETA");
    const int rxy = p->r_xy >= 0 ? p->r_xy : (p->sigma_xy_cells <= 0.0 ? 0 : (int)std::ceil(3.0 * p->sigma_xy_cells));
    const int rth = p->r_theta >= 0 ? p->r_theta : (p->sigma_theta_bins <= 0.0 ? 0 : (int)std::ceil(3.0 * p->sigma_theta_bins));
    if (rxy < 0 || rth < 0 || rxy > LOC_MAX_R_XY || rth > LOC_MAX_R_THETA)
        return noalloc_fail(LOC_ERR_INVALID_ARG, "kernel radius above LOC_MAX_R_XY / LOC_MAX_R_THETA");
    const unsigned int gx = (unsigned int)((p->W + TW - 1) / TW), gy = (unsigned int)((p->H + TH - 1) / TH);
    if ((unsigned long long)gx * gy > kNoAllocMaxBlocks)
        return noalloc_fail(LOC_ERR_INVALID_ARG,
                            "grid too large for the static scratch: ceil(W/32) * ceil(H/16) must be <= 8192");

    NoAllocArgs a{};
    cudaError_t e = scratch_for_current_device(&a.scratch);
    if (e != cudaSuccess) return noalloc_fail(LOC_ERR_CUDA, cudaGetErrorString(e));
    a.B_in = b_in_dev;
    a.B_out = b_out_dev;
    a.occ = occ_dev;
    a.z_out = z_out_dev;
    a.H = p->H;
    a.W = p->W;
    a.K = p->K;
    a.r_xy = rxy;
    a.r_th = rth;
    auto taps = [](double sigma, int r, float* out) {
        if (r == 0 || sigma <= 0.0) {
            for (int d = 0; d <= 2 * r; ++d) out[d] = d == r ? 1.0f : 0.0f;
            return;
        }
        double g[2 * LOC_MAX_R_THETA + 2 * LOC_MAX_R_XY + 1], sum = 0.0;
        for (int d = -r; d <= r; ++d) sum += (g[d + r] = std::exp(-0.5 * (d / sigma) * (d / sigma)));
        for (int d = 0; d <= 2 * r; ++d) out[d] = (float)(g[d] / sum);
    };
    taps(p->sigma_xy_cells, rxy, a.gx);
    taps(p->sigma_theta_bins, rth, a.gt);
    const double px = dx_m / p->cell_m, py = dy_m / p->cell_m;
    for (int k = 0; k < p->K; ++k) {
        const double ang = 2.0 * M_PI * k / p->K;
        const double sx = std::cos(ang) * px - std::sin(ang) * py;
        const double sy = std::sin(ang) * px + std::cos(ang) * py;
        double ox = std::floor(-sx), oy = std::floor(-sy);
        double fx = -sx - ox, fy = -sy - oy;
        if (fx < 1e-9) fx = 0.0;
        if (fx > 1.0 - 1e-9) { fx = 0.0; ox += 1.0; }
        if (fy < 1e-9) fy = 0.0;
        if (fy > 1.0 - 1e-9) { fy = 0.0; oy += 1.0; }
        a.sh[k] = Shift{(int)ox, (int)oy, (float)fx, (float)fy};
    }
    cudaStream_t st = (cudaStream_t)p->stream;
    // the counter must start at zero; a call that stopped early could have left it set
    e = cudaMemsetAsync(&a.scratch->counter, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess) return noalloc_fail(LOC_ERR_CUDA, cudaGetErrorString(e));
    propagate_noalloc_kernel<<<dim3(gx, gy), NT, 0, st>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return noalloc_fail(LOC_ERR_CUDA, cudaGetErrorString(e));
    return LOC_OK;
}
