// Generic fused propagation kernel: Algorithm 1's propagation for all channels plus the Eq. 9
// normaliser, for any kernel radii up to LOC_MAX_R_XY / LOC_MAX_R_THETA and any storage type.
//
// One CTA owns a kGenTH x kGenTW tile of output cells and streams the channels
// kk = -r_th .. K-1+r_th (channel kk mod K; the first and last r_th planes are computed twice
// so that the circular theta blur needs no second pass).  For each channel, in shared memory:
//   raw  = X_{t-1}[c] around the tile, shifted by the channel's integer source offset
//   S    = M * bilinear(raw)                      (Eq. 3 + Algorithm 1's first mask)
//   Xb   = x-blur(S); P[ring] = y-blur(Xb)        (Eq. 7, separable for isotropic Sigma)
// and once the ring holds planes kk-2r_th..kk the output channel o = kk - r_th is
//   X_t[o] = corr * (1/Z_{t-1}) * sum_d gt[d] P[o + d]  (theta blur, Algorithm 1's mask + edge correction)
// The map mask after the blur is folded into corr (0 on occupied cells).  Every thread keeps an
// FP32 running sum of the values it stores (after rounding to the storage type), added
// into an FP64 accumulator once per channel; CTA partials are combined in FP64 by the last
// CTA, which writes Z and advances the log-scale.
#include "kernels.h"

namespace loc {
namespace {

constexpr int TH = kGenTH, TW = kGenTW, NT = 256;
constexpr int RM = LOC_MAX_R_XY, RTM = LOC_MAX_R_THETA;
constexpr int RAW_H = TH + 2 * RM + 1, RAW_W = TW + 2 * RM + 1;
constexpr int S_H = TH + 2 * RM, S_W = TW + 2 * RM;
constexpr int RING = 2 * RTM + 1;
constexpr int CPT = TH * TW / NT;                              // output cells per thread
static_assert(TH * TW % NT == 0, "every thread owns the same number of output cells");

template <typename T>
__global__ void __launch_bounds__(NT) step_generic_kernel(const __grid_constant__ StepArgs a) {
    __shared__ float raw[RAW_H][RAW_W + 1];
    __shared__ float S[S_H][S_W + 1];
    __shared__ float Xb[S_H][TW + 1];
    __shared__ float P[RING][TH][TW + 1];
    __shared__ float Mt[S_H][S_W + 1];
    __shared__ double red[NT / 32];

    const int tid = threadIdx.x;
    const int H = a.H, W = a.W, K = a.K, r = a.r_xy, rt = a.r_th;
    const int ty0 = blockIdx.y * TH, tx0 = blockIdx.x * TW;
    const int sh_h = TH + 2 * r, sh_w = TW + 2 * r;          // S region actually used
    const int rw_h = sh_h + 1, rw_w = sh_w + 1;               // raw region actually used
    const int ring = 2 * rt + 1;

    const int reinit = a.sd->reinit;
    // restart: the input is M / (K n_free); read M and fold 1 / (K n_free) into the scale
    const float in_scale = (reinit ? a.inv_uniform : a.sd->inv_Z) * a.out_mult;
    const T* Bin = static_cast<const T*>(a.B_in);
    T* Bout = static_cast<T*>(a.B_out);

    // map mask around the tile (0 outside the grid)
    for (int q = tid; q < sh_h * sh_w; q += NT) {
        const int jj = q / sh_w, ii = q % sh_w;
        const int j = ty0 - r + jj, i = tx0 - r + ii;
        Mt[jj][ii] = (j >= 0 && j < H && i >= 0 && i < W) ? (float)a.trav[(size_t)j * W + i] : 0.0f;
    }

    KahanF acc;
    float res[CPT];                                            // BF16 residuals of the thread's cells
#pragma unroll
    for (int n = 0; n < CPT; ++n) res[n] = 0.0f;
    for (int kk = -rt; kk < K + rt; ++kk) {
        const int c = ((kk % K) + K) % K;
        const Shift s = a.sh[c];
        const T* plane = Bin + (size_t)c * H * W;
        // raw: rows ty0 - r + oy + [0, rw_h), columns tx0 - r + ox + [0, rw_w)
        for (int q = tid; q < rw_h * rw_w; q += NT) {
            const int jj = q / rw_w, ii = q % rw_w;
            const int j = ty0 - r + s.oy + jj, i = tx0 - r + s.ox + ii;
            float v = 0.0f;
            if (j >= 0 && j < H && i >= 0 && i < W) {
                const size_t o = (size_t)j * W + i;
                v = reinit ? (float)a.trav[o] : Store<T>::ld(plane + o);
            }
            raw[jj][ii] = v;
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
            T* oplane = Bout + (size_t)o * H * W;
            float part = 0.0f;
#pragma unroll
            for (int n = 0; n < CPT; ++n) {                 // the thread's cells, the same every plane
                const int q = tid + n * NT;
                const int j = q / TW, i = q % TW;
                const int gj = ty0 + j, gi = tx0 + i;
                if (gj >= H || gi >= W) continue;
                float v = 0.0f;
                for (int d = -rt; d <= rt; ++d) v += a.gt[d + rt] * P[(o + d + rt) % ring][j][i];
                const size_t off = (size_t)gj * W + gi;
                v = a.corr[off] * in_scale * v;
                part += store_diffused<T>(oplane + off, v, res[n]);
            }
            acc.add(part);
        }
        // the next channel overwrites raw/S/Xb and one ring slot that the theta blur above
        // may still read: wait for every thread first
        __syncthreads();
    }

    const double bt = block_sum<NT>(acc.value(), red);
    const unsigned int nblocks = gridDim.x * gridDim.y;
    SessionDev* sd = a.sd;
    const double log_mult = a.log_out_mult;
    finish_sum<NT>(bt, a.partials, &sd->counter, nblocks, red, [sd, log_mult](double Z) {
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
    });
}

}  // namespace

unsigned int step_num_blocks(int H, int W) {
    return (unsigned int)(((W + TW - 1) / TW) * ((H + TH - 1) / TH));
}

cudaError_t launch_step(const StepArgs& a, int storage, cudaStream_t st) {
    dim3 grid((a.W + TW - 1) / TW, (a.H + TH - 1) / TH);
    switch (storage) {
        case LOC_F32: step_generic_kernel<float><<<grid, NT, 0, st>>>(a); break;
        case LOC_BF16: step_generic_kernel<__nv_bfloat16><<<grid, NT, 0, st>>>(a); break;
        case LOC_F16: step_generic_kernel<__half><<<grid, NT, 0, st>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace loc
