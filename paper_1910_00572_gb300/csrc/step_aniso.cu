// Propagation with anisotropic motion noise (Eq. 5-6 with sigma_x != sigma_y): Algorithm 1
// lines 3-7 for all channels plus the Eq. 9 normaliser, any kernel radii up to LOC_MAX_R_XY /
// LOC_MAX_R_THETA and any storage type.
//
// The motion kernel of output channel k is exp(-1/2 [(d . e_k / sigma_x)^2 + (d . n_k /
// sigma_y)^2 + (dk / sigma_theta)^2]) with e_k the channel's heading phi_k = 2 pi k / K +
// theta_t and n_k its normal, normalised to sum 1: separable into the theta taps and a
// rotated, non-separable x/y stencil that differs per channel.  Since every source plane of
// output channel k is blurred with the same x/y stencil, the theta sum is taken first:
//   S_c   = M * bilinear(X_{t-1}[c])                          (Eq. 3 + Alg. 1 line 4)
//   C_k   = sum_d gt[d] S_{k+d}                               (theta part, circular)
//   T_k   = g_k (x/y) applied to C_k;  G_k = g_k applied to M  (Eq. 7, Eq. 8 for B_0)
//   X_t[k] = M * T_k / G_k * (1 / Z_{t-1})                    (Alg. 1 lines 6-7)
// One CTA owns a kGenTH x kGenTW tile of output cells and streams the source planes
// kk = -r_th .. K-1+r_th through a shared-memory ring over the tile and its halo.  Channel
// k's stencil is computed in the CTA from phi_k (FP32 sin/cos/exp); its normalisation
// cancels in T_k / G_k.
#include "kernels.h"

namespace loc {
namespace {

constexpr int TH = kGenTH, TW = kGenTW, NT = 256;
constexpr int RM = LOC_MAX_R_XY, RTM = LOC_MAX_R_THETA;
constexpr int RAW_H = TH + 2 * RM + 1, RAW_W = TW + 2 * RM + 1;
constexpr int S_H = TH + 2 * RM, S_W = TW + 2 * RM;
constexpr int RING = 2 * RTM + 1;
constexpr int NTAP = (2 * RM + 1) * (2 * RM + 1);

template <typename T>
__global__ void __launch_bounds__(NT) step_aniso_kernel(const __grid_constant__ StepArgs a) {
    __shared__ float raw[RAW_H][RAW_W + 1];
    __shared__ float ring[RING][S_H][S_W + 1];
    __shared__ float C[S_H][S_W + 1];
    __shared__ float Mt[S_H][S_W + 1];
    __shared__ float g[NTAP];
    __shared__ double red[NT / 32];

    const int tid = threadIdx.x;
    const int H = a.H, W = a.W, K = a.K, r = a.r_xy, rt = a.r_th;
    const int ty0 = blockIdx.y * TH, tx0 = blockIdx.x * TW;
    const int sh_h = TH + 2 * r, sh_w = TW + 2 * r;          // S region actually used
    const int rw_h = sh_h + 1, rw_w = sh_w + 1;               // raw region actually used
    const int nring = 2 * rt + 1, side = 2 * r + 1, ntap = side * side;

    const int reinit = a.sd->reinit;
    // restart: the input is M / (K n_free); read M and fold 1 / (K n_free) into the scale
    const float in_scale = (reinit ? a.inv_uniform : a.sd->inv_Z) * a.out_mult;
    const T* Bin = static_cast<const T*>(a.B_in);
    T* Bout = static_cast<T*>(a.B_out);

    for (int q = tid; q < sh_h * sh_w; q += NT) {
        const int jj = q / sh_w, ii = q % sh_w;
        const int j = ty0 - r + jj, i = tx0 - r + ii;
        Mt[jj][ii] = (j >= 0 && j < H && i >= 0 && i < W) ? (float)a.trav[(size_t)j * W + i] : 0.0f;
    }

    KahanF acc;
    for (int kk = -rt; kk < K + rt; ++kk) {
        const int c = ((kk % K) + K) % K;
        const Shift s = a.sh[c];
        const T* plane = Bin + (size_t)c * H * W;
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
        const int slot = (kk + rt) % nring;
        for (int q = tid; q < sh_h * sh_w; q += NT) {
            const int jj = q / sh_w, ii = q % sh_w;
            const float top = gx0 * raw[jj][ii] + fx * raw[jj][ii + 1];
            const float bot = gx0 * raw[jj + 1][ii] + fx * raw[jj + 1][ii + 1];
            ring[slot][jj][ii] = Mt[jj][ii] * (gy0 * top + fy * bot);
        }
        __syncthreads();                    // the theta sum below reads the slot just written
        if (kk >= rt) {
            const int o = kk - rt;
            // channel o's x/y stencil (unnormalised), offsets dj, di in -r..r
            const float phi = a.phi0 + a.dphi * (float)o;
            float sp, cp;
            sincosf(phi, &sp, &cp);
            for (int q = tid; q < ntap; q += NT) {
                const float dj = (float)(q / side - r), di = (float)(q % side - r);
                const float along = (di * cp + dj * sp) / a.sigma_a;
                const float across = (dj * cp - di * sp) / a.sigma_c;
                g[q] = expf(-0.5f * (along * along + across * across));
            }
            // C = theta part over the tile and its halo
            for (int q = tid; q < sh_h * sh_w; q += NT) {
                const int jj = q / sh_w, ii = q % sh_w;
                float v = 0.0f;
                for (int d = -rt; d <= rt; ++d) v += a.gt[d + rt] * ring[(o + d + rt) % nring][jj][ii];
                C[jj][ii] = v;
            }
            __syncthreads();
            T* oplane = Bout + (size_t)o * H * W;
            float part = 0.0f;
            for (int q = tid; q < TH * TW; q += NT) {
                const int j = q / TW, i = q % TW;
                const int gj = ty0 + j, gi = tx0 + i;
                if (gj >= H || gi >= W) continue;
                float v = 0.0f;
                if (Mt[j + r][i + r] > 0.0f) {
                    float t = 0.0f, gm = 0.0f;
                    for (int dj = 0; dj < side; ++dj)
                        for (int di = 0; di < side; ++di) {
                            const float w = g[dj * side + di];
                            t += w * C[j + dj][i + di];
                            gm += w * Mt[j + dj][i + di];
                        }
                    // the stencil's normalisation cancels in t / gm (the theta taps are
                    // normalised); gm >= 1 on a free cell (its own tap is exp(0))
                    v = t / gm * in_scale;
                }
                const size_t off = (size_t)gj * W + gi;
                const uint32_t q_lin = (uint32_t)((size_t)o * H * W + off);
                part += store_out<T>(oplane + off, v, pcg_hash(q_lin ^ a.seed));
            }
            acc.add(part);
        }
        // the next plane overwrites raw, one ring slot, C and the stencil: wait for every thread
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

cudaError_t launch_step_aniso(const StepArgs& a, int storage, cudaStream_t st) {
    if (a.r_xy > RM || a.r_th > RTM || !(a.sigma_a > 0.0f) || !(a.sigma_c > 0.0f)) return cudaErrorInvalidValue;
    dim3 grid((a.W + TW - 1) / TW, (a.H + TH - 1) / TH);
    switch (storage) {
        case LOC_F32: step_aniso_kernel<float><<<grid, NT, 0, st>>>(a); break;
        case LOC_BF16: step_aniso_kernel<__nv_bfloat16><<<grid, NT, 0, st>>>(a); break;
        case LOC_F16: step_aniso_kernel<__half><<<grid, NT, 0, st>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace loc
