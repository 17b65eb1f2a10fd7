/*
 * sdgs.h -- C ABI of libsdgs, a GB300 (sm_103a) renderer for 7D Gaussian Splatting.
 *
 * The render path of 7DGS without adaptive refinement:
 *   sdgs_slice_project  conditional slicing of each 7D Gaussian at (t, d) (Sec. 4.2, Eqs.
 *                       cond_mean / cond_cov, temp_mod / dir_mod; Algorithm 1 steps 3-6) fused
 *                       with the 3DGS perspective (EWA) projection and SH colour (Sec. 4.4).
 *   sdgs_bin_sort       tile binning: one instance per (tile, Gaussian) ordered by
 *                       (tile, depth, Gaussian id) -- the 3DGS tile sort the paper's rasteriser
 *                       uses (Sec. 4.4) -- and per-tile [start, end) ranges.
 *   sdgs_render_fwd     front-to-back alpha compositing per pixel (Sec. 4.4; the 3DGS
 *                       blending rules).
 *   sdgs_render_bwd     adjoint of the three steps above, for the joint optimisation of all 7D
 *                       parameters (Sec. 4.4; Sec. 1 contributions).
 *   sdgs_server_*       a continuous-batching render server over resident scenes.
 *
 * Conventions for every entry point:
 *   - Pointers named "device" are CUDA device memory owned by the caller; the library never
 *     frees them.  Pointers named "host" are ordinary host memory.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Every call only enqueues work on
 *     it and returns, unless it says it synchronises.
 *   - Return value: SDGS_OK or an SDGS_ERR_* code.  On error nothing was enqueued, and
 *     sdgs_last_error() returns a message (thread-local, valid until the next call on the thread).
 *     Errors never trap the device.
 *   - Images are row-major height x width, colour channels innermost (HWC), float32.
 *   - Tiles are 16 x 16 pixels; tiles_x = ceil(width / 16), tiles_y = ceil(height / 16), and
 *     tile_id = ty * tiles_x + tx.
 */
#ifndef SDGS_H_
#define SDGS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum sdgs_status {
  SDGS_OK = 0,
  SDGS_ERR_INVALID_ARG = 1, /* a pointer is NULL, a size is out of range, sh_degree != 3 ... */
  SDGS_ERR_WORKSPACE = 2,   /* workspace missing or smaller than sdgs_bin_workspace_size() */
  SDGS_ERR_OVERFLOW = 3,    /* more (tile, Gaussian) instances than the bins' capacity */
  SDGS_ERR_CUDA = 4,        /* a CUDA runtime call failed; the message names it */
  SDGS_ERR_TIMEOUT = 5,     /* a bounded wait ran out (server; a binning look-back) */
  SDGS_ERR_BUSY = 6,        /* server queue full */
  SDGS_ERR_OOM_BUDGET = 7,  /* a request does not fit the server's memory budget */
  SDGS_ERR_NOT_FOUND = 8    /* unknown scene or request id */
};

#define SDGS_TILE 16
#define SDGS_SH_COEFFS 16

/* A scene of n 7D Gaussians (Sec. 4.1).  All arrays are float32 device memory, C-contiguous.
 *   mean7   [n][7]      mu = (mu_p.x, mu_p.y, mu_p.z, mu_t, mu_d.x, mu_d.y, mu_d.z)
 *   L28     [n][28]     Cholesky factor L of Sigma = L L^T, lower triangle packed row-major:
 *                       L[i][j] (j <= i) at index i*(i+1)/2 + j.  Positive diagonal is the
 *                       caller's responsibility (Sec. 4.1).
 *   opacity [n]         base opacity alpha (already activated, in [0, 1])
 *   sh      [n][16][3]  real SH coefficients of degree 3, index l*l + l + m, RGB innermost
 *   lambda_t, lambda_d  the positive modulation sensitivities of Eqs. temp_mod / dir_mod
 *                       (one scalar each per scene). */
typedef struct sdgs_scene {
  const float* mean7;
  const float* L28;
  const float* opacity;
  const float* sh;
  int64_t n;
  int32_t sh_degree; /* must be 3 */
  float lambda_t;
  float lambda_d;
  int32_t dir_mode;  /* conditioning direction d: 0 = the request's view direction (sdgs_view.d);
                        1 = per Gaussian, the unit vector from the camera centre to its mu_p (the
                        6DGS-style reading of "view direction", Sec. 3); gradients then flow
                        through d into mu_p */
} sdgs_scene;

/* One render request: camera, query time t and conditioning view direction d (Sec. 4.2).
 *   viewmat     world->camera 4x4 row-major, OpenCV axes (+x right, +y down, +z forward)
 *   fx fy cx cy pinhole intrinsics in pixels; pixel (i, j) has its centre at (i + 0.5, j + 0.5)
 *   near_plane  Gaussians whose conditional mean has camera depth < near_plane are culled
 *   t, d[3]     the observed time and unit view direction the 7D Gaussians are conditioned on
 *   bg[3]       background colour added with the final transmittance */
typedef struct sdgs_view {
  float viewmat[16];
  float fx, fy, cx, cy;
  int32_t width, height;
  float near_plane;
  float t;
  float d[3];
  float bg[3];
} sdgs_view;

/* Per-Gaussian screen-space record written by sdgs_slice_project (device, caller-allocated,
 * n entries each; binning takes n < 2^30).  A culled Gaussian has rect = {0, 0, 0, 0}; its other fields are unspecified.
 *   mean2d        [n][2]  projected conditional mean (u, v) in pixels
 *   conic_opacity [n][4]  (a, b, c, alpha_cond): inverse 2D covariance [[a, b], [b, c]] and the
 *                         conditional opacity alpha * f_temp * f_dir
 *   rgb           [n][3]  SH colour max(0, sum beta Y(dir) + 0.5), dir = unit(mu_cond - camera centre)
 *   depth         [n]     camera-space z of mu_cond
 *   rect          [n][4]  uint16 tile rectangle [rx0, rx1) x [ry0, ry1) stored (rx0, ry0, rx1, ry1)
 *   radius        [n]     int32 3-sigma screen radius in pixels (0 when culled) */
typedef struct sdgs_projected {
  float* mean2d;
  float* conic_opacity;
  float* rgb;
  float* depth;
  uint16_t* rect;
  int32_t* radius;
  int64_t n;
} sdgs_projected;

/* Output of sdgs_bin_sort (device, caller-allocated).
 *   tile_keys  [capacity] uint32 tile id of each sorted instance, or NULL to skip writing it
 *   point_list [capacity] uint32 Gaussian id of each sorted instance; instances are ordered by
 *              (tile id, float32 depth, Gaussian id)
 *   ranges     [tiles_x * tiles_y][2] uint32 [start, end) of each tile in the sorted lists;
 *              (0, 0) for a tile without instances
 *   num_instances  device int64: total instance count K written by the call.  It may exceed
 *              capacity; then the lists hold `capacity` of the instances (those of the nearest
 *              Gaussians), still sorted by (tile, depth, id) and covered by the ranges, and
 *              SDGS_ERR_OVERFLOW is reported when the call synchronises.
 *   capacity   number of entries allocated in tile_keys / point_list (< 2^30) */
typedef struct sdgs_bins {
  uint32_t* tile_keys;
  uint32_t* point_list;
  uint32_t* ranges;
  int64_t* num_instances;
  int64_t capacity;
} sdgs_bins;

/* Gradients of sdgs_render_bwd (device, caller-allocated).
 *   dmean7 [n][7], dL28 [n][28], dopacity [n], dsh [n][16][3]
 *   overwrite  0: the call adds (+=) into the arrays, which the caller has zeroed (gradient
 *              accumulation over several renders); nonzero: the call writes every entry (zero for
 *              culled Gaussians) and dlambda, so the arrays need no clearing */
typedef struct sdgs_grads {
  float* dmean7;
  float* dL28;
  float* dopacity;
  float* dsh;
  float* dlambda; /* [2] d/d(lambda_t, lambda_d), added to or written like the others; may be NULL */
  int32_t overwrite;
} sdgs_grads;

/* Library version string, e.g. "sdgs 0.1.0 sm_103a". */
const char* sdgs_version(void);

/* Message of the last error on this thread ("" if none). */
const char* sdgs_last_error(void);

/* Conditional slicing + modulation + culling + EWA projection + SH colour, one pass per Gaussian.
 * Reads the scene (n * 144 bytes of geometry, plus 192 bytes of SH for Gaussians that survive
 * culling) and writes the projected record.  Culled when alpha_cond < 1/255, depth < near_plane,
 * the 2D covariance is not positive definite, or the tile rectangle is empty.
 * Errors: SDGS_ERR_INVALID_ARG (NULL pointer, n < 0, sh_degree != 3, width/height <= 0 or
 * > 65535 * 16, fx/fy <= 0), SDGS_ERR_CUDA (launch failure). */
int sdgs_slice_project(const sdgs_scene* scene, const sdgs_view* view, const sdgs_projected* out,
                       void* stream);

/* Bytes of device workspace sdgs_bin_sort needs for n Gaussians, `capacity` instances and a
 * width x height image.  Writes *bytes (host).  Errors: SDGS_ERR_INVALID_ARG. */
int sdgs_bin_workspace_size(int64_t n, int64_t capacity, int32_t width, int32_t height,
                            size_t* bytes);

/* Tile binning (the 3DGS tile rasteriser of Sec. 3 that Sec. 4.4 renders with).  Sorts the Gaussians by
 * float32 depth (stable, so equal depths keep ascending id), emits in that order one instance per
 * tile of each visible Gaussian's rectangle that the Gaussian may reach, stably sorts the
 * instances by tile id, and writes the per-tile ranges: the result is the stable sort of the
 * 64-bit keys tile_id << 32 | bits(depth) over the kept instances.
 * A tile of the rectangle is dropped only when every pixel centre of the tile has
 * alpha exp(-q/2) < 1/255 by a margin above float32 error; the kept tiles of each tile row form
 * one span.  With conic (a, b, c), opacity alpha and mean (u, v):
 *   det = ac - b^2,  m = 1e-4 + 2^-18 (ac + b^2) / det,  lim = 512 (sqrt^8(255 alpha) - 1) + 1e-3,
 *   Q = lim (1 + 8m) / (1 - m),  hx = sqrt(Q c / det),  hy = sqrt(Q a / det),  dy_r = (-b / c) hx;
 *   row ty is empty when its pixel-centre band [ey0, ey1] = [16 ty + 0.5 - v, 16 ty + 15.5 - v]
 *   misses [-(hy + 0.05 + 2e-3 hy), +(...)]; otherwise, with pad = 0.05 + 2e-3 hx,
 *     x_max = (-b d1 + sqrt(max(aQ - det d1^2, 0))) / a + pad,  d1 = clamp(dy_r, ey0, ey1),
 *     x_min = (-b d2 - sqrt(max(aQ - det d2^2, 0))) / a - pad,  d2 = clamp(-dy_r, ey0, ey1),
 *   and the row keeps ceil((u + x_min - 15.5) / 16) <= tx <= floor((u + x_max - 0.5) / 16);
 *   alpha < 1/255 (lim < 0) drops every tile; det <= 0, m >= 1/2, a <= 0 or a NaN keeps every
 *   tile (a NaN bound keeps the row),
 * every operation a correctly rounded float32 operation in that order, so the kept set is a
 * function of the float32 inputs alone.  Such tiles would composite to the same image.
 * `workspace` is device memory of at least sdgs_bin_workspace_size() bytes, 256-byte aligned.
 * If num_instances_host is not NULL the call synchronises the stream, stores K there and returns
 * SDGS_ERR_OVERFLOW when K > capacity; otherwise it never synchronises (K stays on the device and
 * an overflow only truncates the lists).
 * Every wait inside the sort (a block reading the counts of the blocks before it) is bounded.  If
 * one ever gives up (never expected: a block only waits on blocks that are already running), the
 * later binning kernels skip their work, every tile range is left empty (so compositing reads no
 * list entry) and the device instance count is set to -1: a negative count read back on any path
 * means the frame failed.  With num_instances_host the call then returns SDGS_ERR_TIMEOUT.
 * Errors: SDGS_ERR_INVALID_ARG, SDGS_ERR_WORKSPACE, SDGS_ERR_OVERFLOW, SDGS_ERR_TIMEOUT,
 * SDGS_ERR_CUDA. */
int sdgs_bin_sort(const sdgs_projected* proj, const sdgs_view* view, void* workspace,
                  size_t workspace_bytes, const sdgs_bins* out, int64_t* num_instances_host,
                  void* stream);

/* Binning of `count` (1 to 8) independent problems at once: sdgs_bin_sort of each (projs[j],
 * views[j]) into outs[j] with workspaces[j] (workspace_bytes[j] >= sdgs_bin_workspace_size of that
 * problem), issued as one launch per binning step, each kernel serving every problem (the render
 * server bins the requests it admits together this way).  The results are those of sdgs_bin_sort
 * on each problem alone.  With num_instances_host (host int64[count]) the call synchronises,
 * stores every K and returns the first problem's error if any (SDGS_ERR_OVERFLOW,
 * SDGS_ERR_TIMEOUT); otherwise it only enqueues.  No counterpart in the paper (the serving layer).
 * Errors: SDGS_ERR_INVALID_ARG (count outside [1, 8], a NULL array or a bad problem),
 * SDGS_ERR_WORKSPACE, SDGS_ERR_OVERFLOW, SDGS_ERR_TIMEOUT, SDGS_ERR_CUDA. */
int sdgs_bin_sort_batch(const sdgs_projected* projs, const sdgs_view* views, void* const* workspaces,
                        const size_t* workspace_bytes, const sdgs_bins* outs, int32_t count,
                        int64_t* num_instances_host, void* stream);

/* sdgs_bin_sort without a workspace argument, for callers that cannot allocate device memory --
 * for example a plugin whose host application owns every device allocation, or a latency-bound
 * loop where cudaMalloc's implicit device synchronisation is not acceptable.  The paper has no
 * counterpart: this is a property of the library, not of the method.
 * Same inputs, outputs, ordering and errors as sdgs_bin_sort.  The scratch space is a fixed
 * SDGS_STATIC_BIN_SCRATCH_BYTES (64 MiB) array in the library's device memory, which every GPU
 * that loads the library holds until the process exits.  A problem whose
 * sdgs_bin_workspace_size() exceeds it is rejected with SDGS_ERR_WORKSPACE (nothing enqueued).
 * The first call on each device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current; make that first call before any stream capture.  The call itself allocates
 * nothing.  All calls share the one array: calls whose work overlaps on the GPU (different streams,
 * or host threads without ordering) race and corrupt each other's results.  The looked-up address
 * is cached per device for the life of the process and is not refreshed by cudaDeviceReset: after
 * resetting a device, do not call this function on it again in the same process. */
#define SDGS_STATIC_BIN_SCRATCH_BYTES ((size_t)64 << 20)
int sdgs_bin_sort_static(const sdgs_projected* proj, const sdgs_view* view, const sdgs_bins* out,
                         int64_t* num_instances_host, void* stream);

/* Test support for the sort's bounded waits (no counterpart in the paper).  Runs one stable 8-bit
 * radix pass of the binning sort (digit = key & 255) over n device (key, value) pairs into
 * keys_out / vals_out, with the pass's block tickets starting at first_ticket instead of 0.  With
 * first_ticket = 0 it is an ordinary pass.  With first_ticket > 0 the tiles before first_ticket
 * are never processed, so the blocks that wait on them give up after spin_limit polling rounds
 * (each a short sleep), flag the error and return: the call then returns SDGS_ERR_TIMEOUT.  Every
 * write stays inside keys_out[0, n) / vals_out[0, n).  Synchronises the stream.  `workspace` is
 * device memory of at least sdgs_lookback_selftest_workspace_size() bytes, 256-byte aligned.
 * Errors: SDGS_ERR_INVALID_ARG (n outside [0, 2^30), first_ticket > 2^20, spin_limit outside
 * [1, 2^20]), SDGS_ERR_WORKSPACE, SDGS_ERR_TIMEOUT, SDGS_ERR_CUDA. */
int sdgs_lookback_selftest_workspace_size(int64_t n, size_t* bytes);
/* Test support (no counterpart in the paper): sdgs_bin_sort as if the first pass of its sort had
 * given up waiting (its error bit set before any work), to exercise what every later kernel does
 * then: the lists stay empty, the device instance count becomes -1 and, with num_instances_host,
 * the call returns SDGS_ERR_TIMEOUT.  Same arguments as sdgs_bin_sort. */
int sdgs_bin_sort_failure_selftest(const sdgs_projected* proj, const sdgs_view* view, void* workspace,
                                   size_t workspace_bytes, const sdgs_bins* out, int64_t* num_instances_host,
                                   void* stream);
/* Test support for the span walk's bounded wait (no counterpart in the paper): sdgs_bin_sort of
 * an image of at most 256 tiles per side (span binning) with the span walk's block tickets
 * starting at first_ticket instead of 0 and its look-back giving up after spin_limit polling
 * rounds (each a short sleep).  With first_ticket > 0 the walk blocks before it never run, so the
 * block that waits on them gives up, flags the error and carries on: the lists stay empty, the
 * device instance count becomes -1 and, with num_instances_host, the call returns
 * SDGS_ERR_TIMEOUT.  Every write stays inside the caller's buffers.  Other arguments as
 * sdgs_bin_sort.  Errors: SDGS_ERR_INVALID_ARG (first_ticket > 2^20, spin_limit outside [1, 2^20],
 * an image wider or taller than 256 tiles, or as sdgs_bin_sort), SDGS_ERR_WORKSPACE,
 * SDGS_ERR_TIMEOUT, SDGS_ERR_CUDA. */
int sdgs_span_walk_selftest(const sdgs_projected* proj, const sdgs_view* view, void* workspace,
                            size_t workspace_bytes, const sdgs_bins* out, int64_t* num_instances_host,
                            uint32_t first_ticket, int32_t spin_limit, void* stream);
int sdgs_lookback_selftest(const uint32_t* keys, const uint32_t* vals, uint32_t* keys_out, uint32_t* vals_out,
                           int64_t n, uint32_t first_ticket, int32_t spin_limit, void* workspace,
                           size_t workspace_bytes, void* stream);

/* Measurement support (no counterpart in the paper): one launch of a throughput probe of an SM
 * pipe the rasteriser is bound by, kind 0 = scalar FP32 FMA, 1 = paired FP32 FMA (two FMAs per
 * instruction), 2 = MUFU ex2.approx.  Many independent chains per thread over 64 warps per SM, so
 * the pipe, not latency, limits the rate.  Stores in *ops (host) the operations the launch performs
 * (FLOP for kinds 0 and 1, with an FMA counted as 2; ex2 evaluations for kind 2); the caller times
 * the launch on `stream`.  `sink` is device float32 of at least
 * 8 * 256 * (multiprocessor count) elements (overwritten).  Enqueues only.
 * Errors: SDGS_ERR_INVALID_ARG, SDGS_ERR_WORKSPACE (sink too small), SDGS_ERR_CUDA. */
int sdgs_alu_peak_probe(int32_t kind, int32_t iters, float* sink, int64_t sink_len, double* ops, void* stream);

/* Front-to-back compositing of each 16x16 tile's sorted instances.
 * Per pixel: alpha_i = min(0.99, alpha_cond exp(-1/2 (a dx^2 + c dy^2) - b dx dy)), skipped when
 * below 1/255; the pixel stops before the Gaussian that would take its transmittance below 1e-4.
 * A record whose conic is not positive definite (a <= 0 or ac - b^2 <= 0) is skipped everywhere.
 * Writes image [height][width][3] = sum c_i alpha_i T_i + T_final bg, final_T [height][width] and
 * n_contrib [height][width] (1 + position in the tile list of the last Gaussian blended, 0 if
 * none).  All outputs are device float32 / uint32.  If n_evaluated (device uint64[2]) is not
 * NULL, the number of (pixel, Gaussian) pairs evaluated is ADDED to n_evaluated[0] and the number
 * of those that were blended (contributions) to n_evaluated[1]: the compositing work.
 * Errors: SDGS_ERR_INVALID_ARG, SDGS_ERR_CUDA. */
int sdgs_render_fwd(const sdgs_projected* proj, const sdgs_bins* bins, const sdgs_view* view,
                    float* image, float* final_T, uint32_t* n_contrib, uint64_t* n_evaluated,
                    void* stream);

/* Bytes of device workspace sdgs_render_bwd needs for n Gaussians (per-Gaussian screen-space
 * gradients).  Writes *bytes (host). */
int sdgs_bwd_workspace_size(int64_t n, size_t* bytes);

/* Adjoint of sdgs_render_fwd, sdgs_slice_project (projection, SH, conditioning, modulation and
 * Sigma = L L^T).  Inputs are the forward's scene, view, projected record, bins, final_T and
 * n_contrib, and dL_dimage [height][width][3] (device).  Gradients are added to `grads` (or
 * written, with grads->overwrite).  The culling decisions, radius and tile rectangles are held fixed (they have no derivative); where
 * the 0.99 opacity clamp or the colour clamp at 0 is active the corresponding derivative is 0.
 * `workspace` needs sdgs_bwd_workspace_size() bytes.
 * Errors: SDGS_ERR_INVALID_ARG, SDGS_ERR_WORKSPACE, SDGS_ERR_CUDA. */
int sdgs_render_bwd(const sdgs_scene* scene, const sdgs_view* view, const sdgs_projected* proj,
                    const sdgs_bins* bins, const float* final_T, const uint32_t* n_contrib,
                    const float* dL_dimage, void* workspace, size_t workspace_bytes,
                    const sdgs_grads* grads, void* stream);

/* Densification statistics (Algorithm 1 step 7 and Sec. 4.4), per Gaussian at the view's (t, d):
 *   scale  [n][3]  S = sqrt of the eigenvalues of Sigma_cond (= its singular values), descending
 *   rot    [n][9]  R row-major, columns the matching unit axes (Sigma_cond = R diag(S)^2 R^T),
 *                  last column multiplied by sign(det R) so that det R = +1; the sign of each
 *                  axis is otherwise arbitrary
 *   pt_norm  [n]   |Sigma_pt|, the norm of the space-time coupling block
 *   t_scale  [n]   sqrt(Sigma_t), the temporal scale (time normalised to [0, 1])
 *   split    [n]   uint8: pt_norm > split_pt * extent and t_scale > split_t
 *   prune    [n]   uint8: base opacity < prune_alpha
 * Any output pointer may be NULL (not written).  All device memory, caller-allocated.
 * The paper's thresholds: split_pt = 0.05 (relative to the scene extent), split_t = 0.25,
 * prune_alpha = tau_min = 0.01.  Errors: SDGS_ERR_INVALID_ARG, SDGS_ERR_CUDA. */
typedef struct sdgs_densify_cfg {
  float extent;
  float split_pt;
  float split_t;
  float prune_alpha;
} sdgs_densify_cfg;

typedef struct sdgs_densify {
  float* scale;
  float* rot;
  float* pt_norm;
  float* t_scale;
  uint8_t* split;
  uint8_t* prune;
} sdgs_densify;

int sdgs_densify_stats(const sdgs_scene* scene, const sdgs_view* view, const sdgs_densify_cfg* cfg,
                       const sdgs_densify* out, void* stream);

/* Adaptive Gaussian Refinement (Sec. 4.3, Algorithm 1 steps 1-2).  Four two-layer MLPs
 * Linear(27, 64) -> ReLU -> Linear(64, C_out), C_out = 3, 1, 3, 28, read
 *   f = mu_p (+) mu_t (+) mu_d (+) gamma(t),
 *   gamma(t) = (sin(2^0 pi t), cos(2^0 pi t), ..., sin(2^9 pi t), cos(2^9 pi t)),
 * and add their outputs to mu_p, mu_t, mu_d and the packed L (same packing as L28).  The paper
 * prints the feature, the encoding and the layer sizes; ReLU and the biases are our reading.
 * Weights (device float32, C-contiguous):
 *   w1 [4][64][27], b1 [4][64]   first layers of the MLPs for mu_p, mu_t, mu_d, l (in that order)
 *   w2 [35][64], b2 [35]         output rows 0-2 -> mu_p, 3 -> mu_t, 4-6 -> mu_d, 7-34 -> l; each
 *                                row reads the 64 hidden units of its own MLP */
typedef struct sdgs_agr {
  const float* w1;
  const float* b1;
  const float* w2;
  const float* b2;
} sdgs_agr;

/* Weight gradients, same shapes as sdgs_agr, accumulated (+=). */
typedef struct sdgs_agr_grads {
  float* dw1;
  float* db1;
  float* dw2;
  float* db2;
} sdgs_agr_grads;

/* Refined parameters of every Gaussian at time t: mean7_out [n][7], L28_out [n][28] (device
 * float32, caller-allocated; may not alias the scene's arrays).  The refined scene is then
 * rendered like any other (sdgs_scene pointing at mean7_out / L28_out).
 * Errors: SDGS_ERR_INVALID_ARG, SDGS_ERR_CUDA. */
int sdgs_agr_refine(const sdgs_scene* scene, const sdgs_agr* agr, float t, float* mean7_out, float* L28_out,
                    void* stream);

/* Bytes of device workspace sdgs_agr_refine_bwd needs for n Gaussians. */
int sdgs_agr_bwd_workspace_size(int64_t n, size_t* bytes);

/* Adjoint of sdgs_agr_refine: given dmean7_hat [n][7] and dL28_hat [n][28] (gradients w.r.t. the
 * refined parameters, e.g. from sdgs_render_bwd on the refined scene), accumulates
 * dmean7 += dmean7_hat + (d phi / d mu)^T (...), dL28 += dL28_hat, and the weight gradients.
 * The refinement adds its residual to L without reading L, so the gradient of L28 is dL28_hat
 * itself: dL28 may be NULL, and then the call leaves it to the caller (no copy is made).
 * The weight gradients are summed per block and then across blocks in a fixed order, so repeated
 * calls give identical results.  Errors: SDGS_ERR_INVALID_ARG, SDGS_ERR_WORKSPACE, SDGS_ERR_CUDA. */
int sdgs_agr_refine_bwd(const sdgs_scene* scene, const sdgs_agr* agr, float t, const float* dmean7_hat,
                        const float* dL28_hat, float* dmean7, float* dL28, const sdgs_agr_grads* dagr,
                        void* workspace, size_t workspace_bytes, void* stream);

/* ------------------------------------------------------------------------------------------
 * Render server.  The paper has no serving component; this realises "render requests over
 * resident scenes" on one GPU.  Scenes stay resident (caller-owned device arrays).  Requests --
 * a scene, a view (camera, time t, direction d) and a destination -- enter a FIFO queue and are
 * admitted as soon as a slot (a CUDA stream with its own buffers) is free and the device-memory
 * budget allows: continuous batching, so requests that arrive while others run are admitted while
 * the earlier ones are still on the GPU, and their work overlaps.  Requests admitted together
 * share one batched slicing launch; binning and compositing run on the requests' own streams.
 * Each request's image is bit-identical to rendering it alone through sdgs_slice_project,
 * sdgs_bin_sort and sdgs_render_fwd (no arithmetic depends on the mix).
 * ------------------------------------------------------------------------------------------ */

enum sdgs_request_state {
  SDGS_REQ_QUEUED = 0,
  SDGS_REQ_RUNNING = 1,
  SDGS_REQ_DONE = 2,
  SDGS_REQ_FAILED = 3
};

typedef struct sdgs_server_cfg {
  size_t hbm_budget_bytes;  /* device memory the server may hold for request buffers */
  int32_t max_slots;        /* requests in flight at once (1..64) */
  int32_t queue_capacity;   /* queued requests beyond which submit returns SDGS_ERR_BUSY */
  int32_t device;           /* CUDA device ordinal */
  int32_t batch_window_us;  /* 0: admit requests as soon as a slot is free; > 0: while fewer
                               requests wait than there are free slots, hold admission until the
                               oldest has waited this long, so that they share one batched launch */
} sdgs_server_cfg;

typedef struct sdgs_server_stats {
  uint64_t submitted, completed, failed, retried;
  uint64_t batches;          /* batched slicing launches */
  uint64_t max_batch;        /* largest number of requests in one batched launch */
  uint64_t max_inflight;     /* most requests on the device at the same time */
  size_t bytes_allocated;    /* device memory held by the slots */
} sdgs_server_stats;

typedef struct sdgs_server sdgs_server;

/* Create a server (starts its worker thread; allocates nothing until requests arrive).
 * Errors: SDGS_ERR_INVALID_ARG, SDGS_ERR_CUDA. */
int sdgs_server_create(const sdgs_server_cfg* cfg, sdgs_server** out);

/* Register a resident scene (device arrays stay owned by the caller and must outlive the server).
 * Writes *scene_id.  Errors: SDGS_ERR_INVALID_ARG. */
int sdgs_server_add_scene(sdgs_server* server, const sdgs_scene* scene, int32_t* scene_id);

/* Queue a render of scene_id from `view`.  out_image receives height x width x 3 float32 (HWC)
 * when the request is DONE; it may be device memory or host memory (page-locked host memory keeps
 * the copy asynchronous) and must stay valid until then.  Writes *req_id.
 * Errors: SDGS_ERR_INVALID_ARG, SDGS_ERR_NOT_FOUND (scene), SDGS_ERR_BUSY (queue full),
 * SDGS_ERR_OOM_BUDGET (the request alone needs more than the budget). */
int sdgs_server_submit(sdgs_server* server, int32_t scene_id, const sdgs_view* view,
                       float* out_image, uint64_t* req_id);

/* State of a request and, once DONE, its latency (submit to completion, milliseconds, host
 * monotonic clock).  Errors: SDGS_ERR_NOT_FOUND. */
int sdgs_server_poll(sdgs_server* server, uint64_t req_id, int32_t* state, float* latency_ms);

/* Wait up to timeout_ms for a request to finish.  Returns SDGS_OK when DONE, SDGS_ERR_TIMEOUT if
 * it is still queued or running, or the request's own error code if it FAILED. */
int sdgs_server_wait(sdgs_server* server, uint64_t req_id, int32_t timeout_ms, float* latency_ms);

/* Forget finished requests (their ids become unknown).  Returns the number released. */
int sdgs_server_release(sdgs_server* server, uint64_t req_id);

int sdgs_server_get_stats(sdgs_server* server, sdgs_server_stats* stats);

/* Stop the worker after the requests in flight finish, and free the server's device memory.
 * Queued requests that never started are marked FAILED. */
void sdgs_server_destroy(sdgs_server* server);

#ifdef __cplusplus
}
#endif

#endif /* SDGS_H_ */
