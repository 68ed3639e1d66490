// Host-side launchers of the localizer's kernels (internal to the library).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "loc_dev.cuh"

namespace loc {

// Tile of the generic step kernel (output cells per CTA).
constexpr int kGenTH = 16, kGenTW = 32;

// One propagation of Alg. 1 + the Eq. 9 sum.  `storage` is LOC_F32/LOC_BF16/LOC_F16.
// `partials` must hold step_num_blocks(H, W) doubles.
cudaError_t launch_step(const StepArgs& a, int storage, cudaStream_t st);
unsigned int step_num_blocks(int H, int W);
// The same with anisotropic motion noise (Eq. 5-6, sigma_x != sigma_y): a.phi0, a.dphi,
// a.sigma_a, a.sigma_c give channel k's rotated x/y kernel; a.gx is unused.  Same grid and
// partials as launch_step.
// Dense scan update (dense.cu): the expected-range table, the score of every state (log L
// [K][H][W] and the maximum of log L + log X as an ordered uint) and the reweighting.
cudaError_t launch_range_table(const uint8_t* trav, int H, int W, const float* dirs, int A, float rmax,
                               float inv_step, uint8_t* out, cudaStream_t st);
size_t dense_score_smem(int A, int K, int nu);
cudaError_t launch_dense_score(const uint8_t* table, const uint8_t* trav, const void* B, int storage, int H, int W,
                               int K, int A, const int* m, const float* zs, int nu, float scale, float* logL,
                               unsigned int* maxL, cudaStream_t st);
cudaError_t launch_dense_apply(void* B, int storage, const float* logL, size_t hw, int K, const unsigned int* maxL,
                               float log_mult, double* partials, unsigned int nparts, SessionDev* sd,
                               cudaStream_t st);

// Map difficulty (dense.cu): the probes' table columns and map flags; an argmax of a float
// array (the first index on ties) with its scratch (the arrival counter must start at 0).
cudaError_t launch_gather_columns(const uint8_t* table, const uint8_t* trav, int H, int W, int A,
                                  const int32_t* probes, int n, uint8_t* out, uint8_t* flag, cudaStream_t st);
size_t argmax_f32_scratch_bytes();
cudaError_t launch_argmax_f32(const float* x, size_t n, void* scratch, long long* out, cudaStream_t st);

// Anisotropic propagation (step_aniso.cu).  `tmap` is the tensor map of B_in built by
// make_aniso_tmap, or null (plain loads).
cudaError_t launch_step_aniso(const StepArgs& a, const void* tmap, int storage, cudaStream_t st);
// Whether the TMA input path takes this grid, and its tensor map of one belief buffer.
bool aniso_tma_eligible(int W, int storage);
cudaError_t make_aniso_tmap(void* tmap_out, const void* B, int storage, int H, int W, int K, int r_xy);

// Tiled TMA-pipelined propagation for the default kernel radii (x/y 2, theta 3).  Tile
// configurations are numbered 1 .. step_tiled_num_cfgs(); each needs its own tensor map.
bool step_tiled_eligible(int H, int W, int K, int r_xy, int r_th, int storage);
int step_tiled_num_cfgs();
int step_tiled_default_cfg(int H, int W, int K, int storage);
// Whether tile configuration cfg also writes the argmax of the new tensor (StepArgs::am_idx).
bool step_tiled_fuses_argmax(int cfg);
size_t step_tmap_bytes();
cudaError_t make_step_tmap(void* tmap_out, const void* B, int storage, int H, int W, int K, int cfg);
// Tensor map of a [K][H][W] belief buffer loaded in boxes of box_w x box_h cells of one plane.
cudaError_t make_box_tmap(void* tmap_out, const void* B, int storage, int H, int W, int K, int box_w, int box_h);
cudaError_t launch_step_tiled(const StepArgs& a, const void* tmap, int storage, int cfg, cudaStream_t st);

// ---- Batched propagation (batch.cu): one persistent launch over (session, tile) items of
// many sessions.  Batch configurations 1 .. batch_num_cfgs() are the synchronous tiled
// configurations of the same number (same tile rows, same tensor maps).
struct alignas(128) BatchStatic {           // per session, uploaded once
    unsigned char tmap[2][128];             // tensor maps of B[0], B[1] (CUtensorMap)
    void* B[2];
    const uint8_t* trav;
    const float* corr;
    SessionDev* sd;
    double* partials;                       // >= ntiles doubles
    float inv_uniform, out_mult;
    double log_out_mult;
    int H, W, K, ntx, ntiles, sh_off;       // sh_off: first entry of the session in the shift table
    float g0, g1, g2;
    float gt[7];
};
struct BatchTick {                          // per session, uploaded every tick
    int cur;                                // input buffer
    int pad0, pad1, pad2;
};
struct BatchActive {                        // the sessions propagated this tick, in work order
    int s;                                  // session
    int start;                              // index of its first tile in the tick's work list
};
struct BatchList {
    int n_active;
    int total;                              // tiles of all active sessions
    int pad[2];
};
struct BatchCtl {
    int head;                               // work-queue head (zeroed before every launch)
    int status;                             // LOC_DEV_ERR_* of the launch
};
int batch_num_cfgs();
int batch_tile_rows(int cfg);
// Sets the kernel's shared-memory limit and returns the persistent grid (CTAs per SM x SMs).
cudaError_t batch_prepare(int storage, int cfg, int* grid);
// The per-tick table (device): BatchTick hdr[n] | BatchList | BatchActive act[n] | Shift sh[sum K],
// each part starting on a 16-byte boundary (batch_tick_layout gives the offsets).  Work item q
// of the tick is tile q - act[i].start of session act[i].s for the last i with act[i].start <= q.
// dry != 0 runs every listed tile but leaves partials, Z and the counters untouched.
struct BatchLayout {
    size_t list_off, act_off, shifts_off, bytes;
};
BatchLayout batch_tick_layout(int n_sessions, int sum_k);
cudaError_t launch_batch(int storage, int cfg, int grid, const BatchStatic* ss, const void* tick,
                         const BatchLayout& lay, BatchCtl* ctl, int dry, cudaStream_t st);

// corr[j][i] = trav ? 1 / G(M)(j, i) : 0 with G(M) the x/y blur of M by gx (Eq. 8).
cudaError_t launch_edge_correction(const uint8_t* trav, float* corr, int H, int W,
                                   const float* gx, int r, cudaStream_t st);

// Normalised belief as FP32 [K][H][W].
cudaError_t launch_read_belief(const void* B, int storage, const uint8_t* trav,
                               const SessionDev* sd, float inv_uniform, int H, int W, int K,
                               float* out, cudaStream_t st);

// Belief map over channels: mode LOC_MAP_SUM or LOC_MAP_MAX, FP32 [H][W].
cudaError_t launch_read_marginal(const void* B, int storage, const uint8_t* trav,
                                 const SessionDev* sd, float inv_uniform, int H, int W, int K,
                                 int mode, float* out, cudaStream_t st);

// Argmax of the stored tensor: per-CTA (value, index) pairs then a final pass writing
// out_idx[0] (linear index) and out_val[0] (normalised value).  `scratch` holds
// loc_estimate's results (device): the mass near the argmax state and the strongest cell
// outside its disk (-1 when none holds belief).
struct EstimateOut {
    double mass_near;
    long long second_cell;
    float second_p;
    float pad;
};
// After launch_argmax on the same stream (its index in arg_idx; its scratch reused).
cudaError_t launch_estimate(const void* B, int storage, const uint8_t* trav, const SessionDev* sd,
                            float inv_uniform, int H, int W, int K, void* scratch, const long long* arg_idx,
                            long long r2, int dk, double* partials, unsigned int nparts, EstimateOut* out,
                            cudaStream_t st);
// argmax_scratch_len(n) float + int pairs.
size_t argmax_scratch_bytes(size_t n);
cudaError_t launch_argmax(const void* B, int storage, const uint8_t* trav,
                          const SessionDev* sd, float inv_uniform, int H, int W, int K,
                          void* scratch, long long* out_idx, float* out_val, cudaStream_t st);

// Convert FP32 [K][H][W] to the storage type and set Z = sum of the stored values
// (reinit cleared, logscale unchanged).
cudaError_t launch_set_belief(const float* src, void* B, int storage, size_t n,
                              SessionDev* sd, double* partials, unsigned int nparts,
                              cudaStream_t st);

// ---- LIDAR sample update (lidar.cu)
// m = belief map (max over bins), fs = n_samples / sum(m) (device float).
cudaError_t launch_belief_map(const void* B, int storage, const uint8_t* trav, SessionDev* sd, float inv_uniform,
                              int H, int W, int K, float* m, double* partials, unsigned int nparts,
                              unsigned int* counter, int n_samples, float* fs_out, cudaStream_t st);
// Floyd-Steinberg selection of m * fs -> sel, per-row counts/offsets, total -> *count and (if
// samples) the raster-ordered list of at most cap selected linear indices.  bnd holds
// ((H+31)/32 + 1) * W floats, prog (H+31)/32 + 2 ints.
cudaError_t launch_dither(const float* m, const float* fs, int H, int W, uint8_t* sel, int* rowcnt, int* rowoff,
                          int* count, float* bnd, int* prog, int* status, int cap, int32_t* samples,
                          cudaStream_t st);
cudaError_t launch_ray_ranges(const uint8_t* trav, int H, int W, const int32_t* cells, int n_cells, const float* dirs,
                              int n_dirs, float rmax_cells, float cell_m, float* out, cudaStream_t st);
size_t reweight_scalars_bytes();
// Score the samples against the scan and reweight them (Eq. 9 on the sampled set).
// The map as bits (row j: ceil(W / 32) words, bit b of word w = cell (j, 32 w + b) is free).
cudaError_t launch_pack_bits(const uint8_t* trav, int H, int W, uint32_t* bits, cudaStream_t st);
// bits (from launch_pack_bits, or null) lets the ray casts read a shared-memory window of the map.
cudaError_t launch_score_reweight(void* B, int storage, const uint8_t* trav, const uint32_t* bits, int H, int W, int K,
                                  const int32_t* samples, const int* count, int cap, const float* dirs, int n_dirs,
                                  const int32_t* dir_of, const float* z, int n_used, float rmax_cells, float cell_m,
                                  float inv2s2, float* logL, unsigned int* maxL, void* rs, double* partials,
                                  unsigned int nparts, SessionDev* sd, cudaStream_t st);
// If the session reads as uniform (restart flag), write that belief into B and clear the flag.
cudaError_t launch_materialize(void* B, int storage, const uint8_t* trav, SessionDev* sd, float value,
                               size_t hw, int K, double* partials, unsigned int nparts, cudaStream_t st);

// The bounded-wait limit of the Floyd-Steinberg block hand-offs on the current device, and the
// test hook that makes every hand-off wait on a flag nothing sets (stall != 0).
cudaError_t set_fs_wait(double seconds, int stall);

// Sets the calling thread's error message returned by loc_last_error(NULL).
void set_thread_error(const char* msg);

}  // namespace loc
