/* loc.h -- C-ABI of the GB300 belief-tensor localizer.
 *
 * Method: "Map as The Hidden Sensor: Fast Odometry-Based Global Localization"
 * (Peng & Weikersdorfer, arXiv 1910.00572).  A dense belief tensor B[k][j][i] over the
 * cells (j, i) of an occupancy map and K orientation bins is propagated by odometry
 * (Section III-A, Algorithm 1), corrected by the map (Section III-A.3, Eq. 8), normalised
 * (Eq. 9), and optionally reweighted by LIDAR on Floyd-Steinberg-selected samples
 * (Section III-B).
 *
 * Conventions used by every entry point
 *   - cell (j, i): row j (+y), column i (+x); the cell centre is ((i + 1/2) c, (j + 1/2) c) m.
 *   - bin k: heading k * 2 pi / K + theta_t, where theta_t is the running sum of the w of
 *     every odometry message (Section III-A).
 *   - belief layout: [K][H][W] row-major (channel planes).
 *   - occupancy map: uint8 [H][W] row-major, nonzero = occupied, 0 = free.
 *   - odometry (u, v, w): relative pose between consecutive robot poses, (u, v) metres in
 *     the robot frame at the earlier pose, w radians.
 *
 * Ownership and threading
 *   - The caller owns every host array passed in; the library copies what it keeps
 *     (the map at loc_create).  Readbacks copy into caller buffers and block until done.
 *   - Device memory belongs to the handle.  It comes from the allocator registered with
 *     loc_set_allocator (e.g. a framework's caching allocator), else cudaMalloc.
 *   - All GPU work of a handle runs on the stream given in loc_params.stream (NULL: the
 *     legacy default stream).  Calls that only enqueue work return before it finishes.
 *   - A handle is not thread-safe; distinct handles are independent.
 *
 * Errors
 *   - Every entry point returns a loc_status.  Arguments are validated before any state
 *     changes (a call that fails with LOC_ERR_INVALID_ARG changed nothing).
 *   - A CUDA error or a device-side failure makes the handle sticky-failed: every later call
 *     returns LOC_ERR_STATE until loc_destroy.  loc_last_error(h) describes the failure.
 */
#ifndef LOC_H_
#define LOC_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct loc_session* loc_handle;
typedef struct loc_batch_s* loc_batch;
typedef struct loc_server_s* loc_server;

typedef enum {
    LOC_OK = 0,
    LOC_OK_DEFERRED = 1,       /* loc_step: the Alg. 1 gate was not reached; only theta_t
                                  and the accumulated translation changed */
    LOC_WARN_REINIT = 2,       /* success; since the last report a propagation removed all mass
                                  (Z == 0) and the belief restarted uniform over free cells.
                                  Returned once per new restart count by the calls that
                                  synchronise with the device (loc_sync and the readbacks) */
    LOC_ERR_INVALID_ARG = -1,  /* bad pointer, size, non-finite value, or n mismatch */
    LOC_ERR_OOM = -2,          /* device allocation failed */
    LOC_ERR_CUDA = -3,         /* a CUDA runtime call failed */
    LOC_ERR_TIMEOUT = -4,      /* a bounded device-side wait gave up */
    LOC_ERR_STATE = -5         /* handle is sticky-failed or destroyed */
} loc_status;

/* Belief storage type.  Arithmetic is FP32 in every case.  BF16 stores round by error diffusion
 * along theta: each stored value is one of the two BF16 neighbours of its FP32 value, and the
 * rounding residual of a cell is carried to its next bin, so a cell's mass over its bins is kept
 * to within half a unit in the last place.  FP16 stores the belief times 2^14, rounded to
 * nearest. */
enum { LOC_F32 = 0, LOC_BF16 = 1, LOC_F16 = 2 };
enum { LOC_MAP_SUM = 0, LOC_MAP_MAX = 1 };         /* loc_marginal modes */

#define LOC_MAX_K 256          /* orientation bins per session */
#define LOC_MAX_R_XY 4         /* x/y kernel radius */
#define LOC_MAX_R_THETA 4      /* theta kernel radius */

typedef struct {
    int H, W, K;               /* grid rows, columns, orientation bins (K <= LOC_MAX_K) */
    double cell_m;             /* cell size in metres */
    double sigma_xy_cells;     /* motion-noise std-dev in x and y (cells), Eq. 5-6 */
    double sigma_theta_bins;   /* motion-noise std-dev in theta (bins), Eq. 5-6 */
    int r_xy, r_theta;         /* kernel radii; < 0 selects ceil(3 sigma) */
    double min_shift_cells;    /* Alg. 1 gate |u_{t,k}| >= min_shift (cells); 0: always */
    int storage;               /* LOC_F32 / LOC_BF16 / LOC_F16 */
    int n_samples;             /* Floyd-Steinberg target sample count N_s (Section III-B.1) */
    void* stream;              /* cudaStream_t for all work of the handle, or NULL */
    int kernel;                /* LOC_KERNEL_AUTO, or force LOC_KERNEL_GENERIC / LOC_KERNEL_TILED */
    int tile;                  /* tiled kernel: 0 picks a tile configuration for the grid,
                                  1 .. LOC_TILE_CONFIGS forces one */
    double sigma_cross_cells;  /* anisotropic motion noise (Eq. 6, sigma_x != sigma_y): > 0
                                  sets the sigma across each bin's heading, sigma_xy_cells is
                                  then the sigma along it; the x/y kernel of bin k is rotated
                                  to its heading 2 pi k / K + theta_t, and the default radius is
                                  ceil(3 max(sigma_xy, sigma_cross)).  0 (default) or equal to
                                  sigma_xy_cells: isotropic.  Anisotropic sessions take the
                                  generic-kernel path (kernel must be AUTO or GENERIC) and
                                  cannot join a batch. */
} loc_params;

#define LOC_TILE_CONFIGS 18    /* tile rows x 64 columns, threads: 1: 32 (256), 2: 16 (256),
                                  3: 16 (128), 4: 16 (512), 5: 32 (512); warp-specialised
                                  producer/consumer pipelines: 6: 16 (256), 7: 8 (256),
                                  13: 14 (256); with cells paired 32 columns apart on the
                                  packed FP32 pipe: 8: 16 (128), 9: 16 (256), 10: 32 (256),
                                  11: 8 (128), 12: 16 (128, 2 raw stages); warp-specialised
                                  with the producers split into S-pass and X-pass warps:
                                  14: 16 (320), 15: 14 (288), 16: 28 (512, one CTA per SM);
                                  3 and 2 as a software pipeline over the planes (one CTA
                                  barrier per plane): 17: 16 (128), 18: 16 (256).
                                  With tile = 0 a grid of at least 8 sixteen-row tiles per SM
                                  takes 17 (FP32) or 3 (16-bit storage); smaller grids take
                                  whichever of 6, 15 and 16 gives
                                  the busiest SM the fewest rows to blur (tile rows + 4 per
                                  tile it runs). */

/* Propagation kernel selection: AUTO takes the TMA-tiled kernel when it applies (x/y radius
 * 2, theta radius 3, K >= 8, W a multiple of 16 bytes of storage) and the generic one
 * otherwise; forcing TILED where it does not apply fails loc_create with INVALID_ARG. */
enum { LOC_KERNEL_AUTO = 0, LOC_KERNEL_GENERIC = 1, LOC_KERNEL_TILED = 2 };

/* Fill *p with the defaults: sigma_xy 0.5 cells, sigma_theta 1 bin, radii ceil(3 sigma),
 * min_shift 0, LOC_F32, n_samples 4096, NULL stream, LOC_KERNEL_AUTO, tile 0.  H, W, K,
 * cell_m are set to 0. */
void loc_params_default(loc_params* p);

/* Optional device allocator for every later loc_create.  alloc(bytes, stream, ctx) returns
 * a device pointer or NULL; release(ptr, stream, ctx) frees it.  Pass NULLs to go back to
 * cudaMalloc/cudaFree.  Not thread-safe with concurrent loc_create/loc_destroy. */
typedef void* (*loc_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*loc_free_fn)(void* ptr, void* stream, void* ctx);
void loc_set_allocator(loc_alloc_fn alloc, loc_free_fn release, void* ctx);

/* Create a session on the current CUDA device.  occ: host uint8 [H][W] (copied).
 * The initial belief is uniform over free cells (Section III-A: the initial state is
 * unknown).  Precomputes G(B_0)^-1 of Algorithm 1's edge correction (Eq. 8) on the device.
 * Errors: INVALID_ARG (sizes <= 0, K > LOC_MAX_K, radii above the maxima, cell_m <= 0,
 * no free cell), OOM, CUDA.  On error *out is NULL. */
loc_status loc_create(const uint8_t* occ, const loc_params* p, loc_handle* out);

/* One odometry message (Section III-A, Eq. 2, Algorithm 1).  theta_t += w and the
 * translation accumulates; when |accumulated| / cell >= min_shift the whole tensor is
 * propagated on the device: per-channel bilinear shift (Eq. 3), map mask, 3-D Gaussian
 * blur (Eq. 5-7), map mask, edge normalisation (Eq. 8), then the normaliser Z = sum B
 * (Eq. 9) is reduced in FP64 and applied lazily.  If Z == 0 the belief restarts uniform
 * over free cells (counted in loc_stats).  Returns LOC_OK (work enqueued, asynchronous) or
 * LOC_OK_DEFERRED.  Errors: INVALID_ARG (non-finite input), STATE, CUDA. */
loc_status loc_step(loc_handle h, double u, double v, double w);

/* LIDAR sample update (Section III-B, Eq. 9).  ranges: host float[n_beams] in metres,
 * beam b at angle_min + b * angle_inc relative to the robot heading.  Beams with
 * b % beam_stride == 0 and range < r_max are scored with a Gaussian range likelihood of
 * std-dev sigma_r against the expected range of every sampled state, found by walking the
 * grid from the cell centre along the beam to the first occupied cell or the grid edge
 * (capped at r_max).  Samples are the cells that Floyd-Steinberg dithering selects from the
 * belief map (max over channels) scaled to about loc_params.n_samples selections
 * (Section III-B.1); every channel of a sampled cell is a sampled state.  The sampled states
 * are multiplied by their likelihood and renormalised so that the set keeps its total
 * mass (Eq. 9's eta over the sampled set); other states are unchanged.  Enqueued on the
 * handle's stream (asynchronous).  Errors: INVALID_ARG (sizes, non-finite values,
 * sigma_r <= 0, r_max <= 0, beam_stride < 1), STATE, CUDA. */
loc_status loc_lidar_update(loc_handle h, const float* ranges, int n_beams, double angle_min,
                            double angle_inc, double r_max, int beam_stride, double sigma_r);

/* Same as loc_lidar_update but with the sampled cells given by the caller: host int32
 * linear indices j * W + i, no duplicates, at most H * W of them (e.g. from a previous
 * loc_samples call, or from another sampler).  Synchronous for the host array. */
loc_status loc_lidar_update_cells(loc_handle h, const int32_t* cells, int n_cells,
                                  const float* ranges, int n_beams, double angle_min,
                                  double angle_inc, double r_max, int beam_stride,
                                  double sigma_r);

/* The cells selected by the last loc_lidar_update (host int32 linear indices j * W + i in
 * raster order; the paper's "samples from the belief map", Fig. 1c).  *n receives the count;
 * at most cap indices are written.  Synchronous. */
loc_status loc_samples(loc_handle h, int32_t* out, size_t cap, int* n);

/* Floyd-Steinberg dithering of a caller map (Section III-B.1), as loc_lidar_update applies it
 * to the belief map: value v = min(1, m[q] * fs) plus the diffused error, selected iff
 * >= 0.5, errors 7/16 right, 3/16 down-left, 5/16 down, 1/16 down-right, raster order, all in
 * FP32 with the operations in that order (no fused multiply-add).  m: host float[H][W] of
 * the handle's grid; sel: host uint8[H][W] (1 = selected); *count receives the number of
 * selected cells.  Synchronous. */
loc_status loc_dither(loc_handle h, const float* m, float fs, uint8_t* sel, int* count);

/* Expected ranges (metres) used by the LIDAR likelihood, for given cells and unit directions:
 * out[c * n_dirs + d] = distance from the centre of cell cells[c] along dirs[2d], dirs[2d+1]
 * (FP32 cos, sin in the map frame) to the first occupied cell or the grid edge, capped at
 * r_max; a tie between the next x and y cell boundaries steps x first; FP32 arithmetic in
 * a fixed order (no fused multiply-add).  Host arrays; synchronous. */
loc_status loc_ray_ranges(loc_handle h, const int32_t* cells, int n_cells, const float* dirs,
                          int n_dirs, double r_max, float* out);

/* The pose estimate and how concentrated the belief is around it (Section III-A.3's belief
 * map; the multiple hypotheses of Section V).  The estimate is loc_argmax's state (k, j, i):
 * pose x = (i + 1/2) cell_m, y = (j + 1/2) cell_m, theta = 2 pi k / K + theta_t mod 2 pi,
 * belief p.  mass_near = the belief of the states whose cell lies within radius_m of (j, i)
 * (dj^2 + di^2 <= floor(radius_m^2 / cell_m^2 + 1e-9), so a radius of a whole number of cells
 * includes the cells at that distance) and whose bin is within dk of k (circular).  The second
 * hypothesis is the largest belief-map value (max over bins) among the cells outside that disk,
 * the lowest cell index on ties: (second_j, second_i, second_p), or (-1, -1, 0) when no cell
 * outside holds belief; second_ratio = second_p / p.  Synchronous.
 * Errors: INVALID_ARG (null out, radius_m negative or not finite, dk < 0), OOM, CUDA, STATE. */
typedef struct loc_estimate_t {
    int k, j, i;
    double x, y, theta, p;
    double mass_near;
    int second_j, second_i;
    double second_p, second_ratio;
} loc_estimate_t;
loc_status loc_estimate(loc_handle h, double radius_m, int dk, loc_estimate_t* out);

/* Readbacks (synchronous).  n must equal the element count exactly.
 *   loc_belief:   normalised belief, host float[K][H][W].
 *   loc_marginal: host float[H][W]: LOC_MAP_MAX = max over channels (the paper's belief
 *                 map, Section III-A.3), LOC_MAP_SUM = sum over channels (marginal).
 *   loc_argmax:   the most probable state (k, j, i) and its probability; ties go to the
 *                 lowest linear index in [K][H][W] order.  After a loc_step through a
 *                 warp-specialised tile configuration (6, 7, 13-16) the step kernel has
 *                 already combined this argmax, and the call only reads it back; otherwise
 *                 it makes one pass over the tensor. */
loc_status loc_belief(loc_handle h, float* out, size_t n);
loc_status loc_marginal(loc_handle h, float* out, size_t n, int mode);
loc_status loc_argmax(loc_handle h, int* k, int* j, int* i, float* p);

/* Replace the belief by host float[K][H][W] (non-negative, finite, positive sum); it is
 * normalised on the device.  Synchronous.  Values on occupied cells are kept as given. */
loc_status loc_set_belief(loc_handle h, const float* b, size_t n);

/* Session scalars (synchronous): theta_t, the last normaliser Z, the running log-scale
 * sum(log Z), the number of propagations and of restarts after Z == 0. */
loc_status loc_stats(loc_handle h, double* theta_t, double* last_Z, double* logscale,
                     long long* n_propagations, long long* n_reinit);

/* Allocation-free propagation (the paper has no counterpart: this is a deployment aid).
 * For callers that must not allocate device memory while they run: real-time loops where a
 * cudaMalloc could stall, certified or embedded stacks whose memory is fixed at start-up,
 * and hosts whose allocator belongs to another runtime.  The caller owns every buffer:
 *   occ_dev    device uint8 [H][W], nonzero = occupied;
 *   b_in_dev   device float [K][H][W], the belief to propagate (used as given);
 *   b_out_dev  device float [K][H][W], receives the propagated, unnormalised tensor: the
 *              same shift, map mask, motion blur and edge correction as loc_step, without
 *              the division by Z;
 *   z_out_dev  device double, receives Z = the sum of b_out;
 *   dx_m, dy_m translation in metres in the frame of bin 0 (bin k moves by R(2 pi k / K)).
 * From p it uses H, W, K, cell_m, the sigmas and radii and stream; storage must be LOC_F32
 * and the noise isotropic (sigma_cross_cells 0 or equal to sigma_xy_cells).
 * The only other memory it touches is a 64 KiB + 256 B scratch array compiled into the
 * library, which every GPU that loads the library keeps until the process exits.  That
 * bounds the grid: ceil(W / 32) * ceil(H / 16) must be <= 8192 (e.g. 2048 x 2048 cells);
 * larger grids are rejected with LOC_ERR_INVALID_ARG.  It never calls cudaMalloc, cudaFree
 * or any allocating routine.  The first call on a device looks up that device's scratch
 * address, so make it before any stream capture.  All calls on a device share the one
 * scratch array: calls whose kernels overlap on the GPU race and give wrong results.
 * Asynchronous on p->stream.  Errors: INVALID_ARG, CUDA; message in loc_last_error(NULL). */
loc_status loc_propagate_noalloc(const loc_params* p, const uint8_t* occ_dev,
                                 const float* b_in_dev, float* b_out_dev, double* z_out_dev,
                                 double dx_m, double dy_m);

/* ---- Dense scan update: Eq. 9 on every state from a precomputed expected-range table.
 *
 * The map is static, so the expected range of every cell along n_angles fixed directions
 * 2 pi a / n_angles can be cast once (Section III-B's ray model, the same FP32 grid walk as
 * the sampled update) and stored in 8 bits.  A scan then scores every (cell, bin) state from
 * that table and reweights the whole tensor, the dense limit of Eq. 9 (no dithering). */

#define LOC_MAX_TABLE_DIRS 1440    /* table directions per session */
#define LOC_MAX_DENSE_BEAMS 2048   /* used beams (every beam_stride-th, range < r_max) per scan */

/* Builds (or rebuilds) the session's table: code (a, j, i) = floor(t * inv_step + 0.5)
 * capped at 255, t = the FP32 walk from the centre of cell (j, i) along direction a in cells,
 * capped at float(r_max / cell_m), inv_step = float(255 / that cap); each FP32 operation
 * rounded.  The code stands for code * float(r_max / 255) metres; occupied cells hold 0.
 * n_angles: a positive multiple of K, <= LOC_MAX_TABLE_DIRS (bin k's heading is direction
 * k n_angles / K).  r_max (m) > 0: the range cap, also the dropout threshold of the dense
 * update.  Allocates n_angles * H * W bytes on the device; synchronous.
 * Errors: INVALID_ARG, OOM, CUDA, STATE. */
loc_status loc_range_table(loc_handle h, int n_angles, double r_max);

/* Copies the table, [n_angles][H][W] uint8, to `out` (n = n_angles * H * W); synchronous.
 * Errors: INVALID_ARG (no table, or n mismatch), CUDA, STATE. */
loc_status loc_range_table_read(loc_handle h, uint8_t* out, size_t n);

/* Dense scan update (Eq. 9 on every state).  ranges: host float[n_beams] in metres, finite,
 * >= 0; beam b of a state in bin k points at 2 pi k / K + theta_t + angle_min + b angle_inc
 * and reads table direction (k n_angles / K + m_b) mod n_angles, where
 * m_b = floor((theta_t + (angle_min + angle_inc b)) / (2 pi / n_angles) + 0.5) mod n_angles
 * (FP64, host).  Used beams: b % beam_stride == 0 and range < the table's r_max (at most
 * LOC_MAX_DENSE_BEAMS).  log L = -sum over used beams of (z_b - code * step)^2 / (2 sigma_r^2)
 * for every state (FP32); the tensor becomes b w / sum(b w) with w = exp(log L - max), the
 * maximum over the states of free cells, and the log-scale grows by log(sum(b w)) + max.  No
 * used beam: no change.  Allocates K * H * W floats of scratch on first use.  Asynchronous
 * on the session's stream.  Errors: INVALID_ARG (including no table), OOM, CUDA, STATE. */
loc_status loc_lidar_update_dense(loc_handle h, const float* ranges, int n_beams, double angle_min,
                                  double angle_inc, int beam_stride, double sigma_r);

/* Map difficulty D_M (Eq. 11) on probe cells through the dense scorer.  For each probe
 * (a free cell, linear index j W + i), its noise-free scan is read off the range table: beams
 * on table directions probe_bin n_angles / K + b beam_step (mod n_angles), b beam_step <
 * n_angles, each range the table's code at the probe (code 255, the capped range, skipped).
 * Every state is scored against it as in loc_lidar_update_dense (sigma_r), and the best match
 * is the argmax of log L over the states of free cells (the first in [K][H][W] order on ties);
 * e_p = cell_m * |p - p_hat| between cell centres.  errors (may be NULL): double[n_probes]
 * receives e_p; *n_wrong = the number of probes with e_p > c_m, so D_M is estimated as
 * n_wrong / n_probes.  Needs the range table; leaves the belief unchanged; synchronous.
 * Errors: INVALID_ARG (no table, probe out of grid or occupied, bad parameters), OOM, CUDA,
 * STATE. */
loc_status loc_map_difficulty(loc_handle h, const int32_t* probes, int n_probes, int probe_bin,
                              int beam_step, double sigma_r, double c_m, double* errors, int* n_wrong);

/* ---- Batched propagation of many sessions (one persistent launch per tick).
 * Algorithm 1's propagation and the Eq. 9 normaliser for every session whose gate opens, over a work
 * list of (session, tile) items that the launch's CTAs take from a device queue; the CTA that
 * finishes a session's last tile sums that session's tile partials into Z in the same fixed
 * order as loc_step's tiled kernel with the same tile configuration, so a session's result
 * does not depend on the other sessions of the batch. */
#define LOC_BATCH_CONFIGS 3    /* the synchronous tile configurations 1-3 of LOC_TILE_CONFIGS */

/* Group n sessions (distinct handles on one device, one storage type, one stream, each able to
 * use the tiled kernel: default radii, K >= 8, W a multiple of 4 (FP32) or 8 (16-bit)).  The
 * batch does not own the sessions: destroy it before any of them.  tile: 0 = autotune (every
 * configuration runs the whole batch in a dry run that leaves the sessions unchanged, the
 * fastest is kept and remembered for this storage type and multiset of (H, W, K)), or
 * 1 .. LOC_BATCH_CONFIGS.  use_graph != 0 captures the tick (host-to-device copy of the
 * per-tick table, queue reset, kernel) in CUDA graphs, one launch per tick.  The batch runs on
 * a stream of its own, ordered after and before the sessions' stream by events.
 * Synchronous.  Errors: INVALID_ARG, STATE, OOM, CUDA. */
loc_status loc_batch_create(const loc_handle* sessions, int n, int tile, int use_graph, loc_batch* out);

/* One tick: u, v, w are host double[n], the odometry increments of the sessions in creation
 * order (as loc_step takes them).  Each session's gate is evaluated as in loc_step; the
 * sessions that pass are propagated together.  *n_moved (may be NULL) receives their number.
 * Returns LOC_OK (work enqueued, asynchronous) or LOC_OK_DEFERRED (no session moved, nothing
 * launched).  The host tables use two pinned buffers, so a call waits for the tick before the
 * previous one.  Single-session calls on the same handles may be mixed in between ticks.
 * Errors: INVALID_ARG (changes nothing), STATE, CUDA (fails the batch and its sessions). */
loc_status loc_batch_step(loc_batch b, const double* u, const double* v, const double* w, int* n_moved);

/* Wait for the batch's work; returns the first device-side error of the launches or of a
 * session. */
loc_status loc_batch_sync(loc_batch b);

/* The tile configuration in use, the number of work items, the persistent grid (CTAs), and
 * the autotuner's mean dry-run milliseconds per configuration (float[LOC_BATCH_CONFIGS], 0
 * where not timed).  Any pointer may be NULL. */
loc_status loc_batch_info(loc_batch b, int* tile, int* n_items, int* grid, float* tune_ms);

/* Free the batch (waits for its work; the sessions stay).  b may be NULL. */
loc_status loc_batch_destroy(loc_batch b);

/* Description of the batch's last failure ("" if none; b may be NULL). */
const char* loc_batch_last_error(loc_batch b);

/* Device bytes a session created with p holds once it has run a LIDAR update (the belief
 * tensors, map, correction, reduction and sampling scratch, each allocation rounded up to
 * 512 bytes).  Used for admission against a memory budget.  No device work. */
loc_status loc_session_bytes(const loc_params* p, size_t* bytes);

/* ---- Serving loop: many robot sessions stepped as their messages arrive (continuous batching).
 * Sessions are opened against a device-memory budget (loc_session_bytes each) and admitted
 * first come, first served as memory frees up.  Odometry and scan messages may be submitted
 * from any thread; each session's messages are applied in submission order.  A worker thread
 * forms a tick from whatever sessions have work.  Per session, in message order: odometry
 * messages run through its Alg. 1 gate one by one; at most one scan message runs in the tick
 * (on the session's stream, before the tick's batched launch, which waits for it); the first
 * odometry message that opens the gate joins the tick's batched launch and ends the session's
 * share of the tick (a scan after it waits for the next tick).  So the propagation points and every
 * result depend only on the session's own message stream, never on the load: a session gives
 * the same belief served alone or in any mix (with the same tile configuration).  A completion
 * thread timestamps finished work for the latency statistics. */
#define LOC_SESSION_PENDING 0      /* waiting for admission */
#define LOC_SESSION_ACTIVE 1
#define LOC_SESSION_CLOSED 2
#define LOC_SESSION_FAILED 3

typedef struct {
    double hbm_budget_bytes;       /* device bytes all admitted sessions may hold together */
    int storage;                   /* belief storage of every session (LOC_F32/BF16/F16) */
    int batching;                  /* 1: one persistent batched launch per tick (default);
                                      0: one loc_step per odometry message (the plain path) */
    int tile;                      /* batch tile configuration; 0 = autotune on the first batch
                                      and keep it */
    int use_graph;                 /* capture each tick in a CUDA graph (default 1) */
    int n_streams;                 /* streams for scan updates and plain steps (default 32);
                                      each tick hands them out in turn, a session's work on a
                                      new stream waiting for its work on the previous one.  The
                                      device runs at most CUDA_DEVICE_MAX_CONNECTIONS streams at
                                      once (CUDA's default is 8; set it to 32 in the environment
                                      before the process's first CUDA call) */
} loc_server_params;

typedef struct {
    int n_active, n_pending, n_closed, n_failed;    /* sessions by state */
    double bytes_used, bytes_budget;
    long long n_ticks;             /* worker iterations that launched work */
    long long n_messages;          /* messages fully processed */
    long long n_propagations, n_scans;
    double cell_updates;           /* sum of K * H * W over the propagations */
    double mean_batch;             /* propagations per batched launch */
    double step_p50_ms, step_p99_ms, step_max_ms;   /* odometry message arrival (the one that
                                      opened the gate) to the end of its propagation */
    double scan_p50_ms, scan_p99_ms, scan_max_ms;   /* scan arrival to the end of its update */
    double first_s, last_s;        /* server clock of the first arrival and last completion */
    /* Where the time goes.  Device time is measured between CUDA events recorded where each
     * piece of work could begin (after its ordering waits) and where it ends, so work that
     * overlaps on the device is counted once per piece. */
    double batch_device_ms;        /* sum over batched launches (table copy + kernel) */
    double batch_alg_bytes;        /* their algorithmic HBM bytes: 2 x storage bytes per
                                      cell-update plus 5 bytes of map fields per map cell */
    long long n_batches;
    double scan_device_ms;         /* sum over scan updates (belief map, dithering, ray casts,
                                      scoring and reweighting) */
    long long n_scans_timed;
    double plain_device_ms;        /* sum over plain-path propagations (one loc_step each) */
    double plain_alg_bytes;
    long long n_plain;
    double host_gather_ms;         /* worker thread: taking work from the queues (gate included) */
    double host_batch_ms;          /* worker thread: preparing and launching the batched tick */
    double host_scan_ms;           /* worker thread: the scan phase of the ticks (host work and
                                      launches of the scan updates, up to the last one issued) */
    double host_plain_ms;          /* worker thread: the plain-path loc_step calls */
} loc_server_stats_t;

void loc_server_params_default(loc_server_params* p);
/* Start a server (its worker and completion threads) on the current device.  Errors:
 * INVALID_ARG, CUDA. */
loc_status loc_server_create(const loc_server_params* p, loc_server* out);
/* Open a session: the map and parameters as loc_create takes them (storage and stream are the
 * server's).  *id receives its id; it starts LOC_SESSION_PENDING and is admitted when its
 * loc_session_bytes fit in the budget next to the admitted sessions and every earlier pending
 * session is admitted.  Messages may be submitted at once; they run after admission.
 * INVALID_ARG when the parameters are invalid, the map has no free cell, the session can never
 * fit the budget, or a batched server gets a session the tiled kernel cannot take. */
loc_status loc_server_open(loc_server s, const uint8_t* occ, const loc_params* p, int* id);
/* Close a session after its queued messages: its memory returns to the budget. */
loc_status loc_server_close(loc_server s, int id);
/* n odometry messages: session ids[i] moved by (u[i], v[i], w[i]) as loc_step takes them, at
 * t_arrival[i] seconds of loc_server_now (NULL: now).  Non-finite values or unknown/closed ids
 * fail the whole call (INVALID_ARG) before any message is queued. */
loc_status loc_server_odometry(loc_server s, int n, const int* ids, const double* u, const double* v,
                               const double* w, const double* t_arrival);
/* A scan message for session id (arguments as loc_lidar_update; the ranges are copied);
 * t_arrival < 0 means now. */
loc_status loc_server_scan(loc_server s, int id, const float* ranges, int n_beams, double angle_min,
                           double angle_inc, double r_max, int beam_stride, double sigma_r, double t_arrival);
/* Seconds since the server started (steady clock). */
double loc_server_now(loc_server s);
/* Wait until every pending session that fits the budget is admitted, every submitted message
 * of the admitted sessions is processed and its device work has finished (sessions that must
 * wait for memory are not waited for).  TIMEOUT after timeout_s seconds. */
loc_status loc_server_drain(loc_server s, double timeout_s);
loc_status loc_server_stats(loc_server s, loc_server_stats_t* out);
/* Clear the counters and latency samples (not the sessions). */
loc_status loc_server_reset_stats(loc_server s);
/* State of session id and its handle (NULL unless active).  Readbacks through the handle are
 * valid only while no message of that session is queued or running, e.g. after
 * loc_server_drain. */
loc_status loc_server_session(loc_server s, int id, int* state, loc_handle* h);
/* Stop the threads (messages still queued are dropped), wait for the device work in flight
 * and free every session.  s may be NULL. */
loc_status loc_server_destroy(loc_server s);
const char* loc_server_last_error(loc_server s);

/* ---- Test hook of the bounded device waits (no paper counterpart).
 * Every device-side wait of the library gives up after a limit, records LOC_DEV_ERR_TIMEOUT in
 * the session's status and returns, so a stalled hand-off surfaces as LOC_ERR_TIMEOUT (after
 * which the handle fails with LOC_ERR_STATE) while the CUDA context stays usable.  This hook
 * exercises that path on the Floyd-Steinberg block hand-offs of the scan update, whose waits
 * poll a progress flag in global memory: with stall != 0 every hand-off waits on a flag that
 * nothing sets, so each wait runs for wait_limit_s and gives up; the sample list of that scan is
 * empty.  stall = 0, wait_limit_s = 0.2 restore the defaults.  Applies to the current device,
 * process-wide; not for use while other threads run scan updates.
 * Errors: INVALID_ARG (wait_limit_s outside (0, 10]), CUDA. */
loc_status loc_debug_fs_stall(int stall, double wait_limit_s);

/* Wait for all enqueued work of the handle; returns the first device-side error if any. */
loc_status loc_sync(loc_handle h);

/* Free the session (waits for its work).  h may be NULL. */
loc_status loc_destroy(loc_handle h);

/* Human-readable description of the last failure of h (or of the calling thread when h is
 * NULL).  Valid until the next call on the same handle / thread. */
const char* loc_last_error(loc_handle h);

#ifdef __cplusplus
}
#endif
#endif /* LOC_H_ */
