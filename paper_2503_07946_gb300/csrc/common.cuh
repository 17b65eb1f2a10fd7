// Shared definitions of the CUDA path (kernels and C-ABI glue).  Nothing here is used by the
// oracle.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sdgs.h"

namespace sdgs {

// Programmatic dependent launch.  A kernel started by launch_pdl may be scheduled while the
// kernel before it in the stream is still finishing; it calls griddep_wait() before it touches
// global memory, which returns once that kernel has completed and its writes are visible (and is
// a no-op after an ordinary launch).  This hides the launch gap between the dependent kernels of
// one render.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

constexpr int kTile = 16;
constexpr int kTilePixels = kTile * kTile;
constexpr float kAlphaMin = 1.0f / 255.0f;  // compositing skip threshold and cull threshold
constexpr float kAlphaMax = 0.99f;          // opacity clamp per pixel
constexpr float kTMin = 1e-4f;              // transmittance stop threshold
constexpr float kDilation = 0.3f;           // added to the 2D covariance diagonal
constexpr float kJacClamp = 1.3f;           // x/z, y/z clamp (in units of tan(fov/2)) for J
constexpr float kExtent = 3.0f;             // radius = ceil(3 sqrt(lambda_max))

// Error reporting (api.cu).
void set_error(const char* fmt, ...);
int cuda_status(cudaError_t e, const char* what);

inline int tiles_of(int px) { return (px + kTile - 1) / kTile; }

// Multiprocessor count of the current device (cached per device), for grid sizing.
int device_sm_count();

// Internal launchers (one .cu each).
cudaError_t launch_slice_project(const sdgs_scene& s, const sdgs_view& v, const sdgs_projected& o,
                                 cudaStream_t st);

// Slicing of several requests (the server's): up to 8 per launch, each launch's arguments passed
// by value; the same kernel as a single request, so the same results.
constexpr int kMaxBinBatch = 8;
struct SliceRequest {
  sdgs_scene scene;
  sdgs_view view;
  sdgs_projected out;
};
cudaError_t launch_slice_project_batch(const SliceRequest* reqs, int count, cudaStream_t st);

struct BinPlan {
  int64_t n;
  int64_t capacity;
  int num_tiles;
  int tile_bits;
  bool spans;    // row-span binning (both tile counts <= 256); else instance records and a tile sort
  int row_bits;  // span binning: bits of the row sort
  // workspace carve-up (byte offsets)
  size_t off_dkeys[2], off_dvals[2], off_first, off_ikeys[2], off_ivals, off_err, off_sort_d, off_sort_t,
      off_partials, total;
  size_t off_svals, off_walk, off_ctab, off_rowtot;  // span binning only
  int64_t partial_cap;  // entries available for scan partials
};
BinPlan plan_bins(int64_t n, int64_t capacity, int width, int height);
// inject_err != 0 (test support only) starts the sort's error word at that value.
cudaError_t launch_bin_sort(const sdgs_projected& p, const sdgs_view& v, const BinPlan& plan,
                            char* ws, const sdgs_bins& out, cudaStream_t st, uint32_t inject_err = 0,
                            uint32_t walk_ticket = 0, int spin_limit = 0);

// Binning of up to kMaxBinBatch requests with one launch per step (each kernel serves request
// blockIdx.y); the same results as binning each request on its own.
struct BinRequest {
  sdgs_projected proj;
  sdgs_view view;
  BinPlan plan;
  char* ws;
  sdgs_bins out;
  uint32_t inject_err;
  // test support: the span walk's block tickets start here, and its waits give up after this
  // many polling rounds (0: the default)
  uint32_t walk_ticket = 0;
  int spin_limit = 0;
};
cudaError_t launch_bin_sort_batch(const BinRequest* reqs, int count, cudaStream_t st);
size_t lookback_selftest_bytes(int64_t n);
cudaError_t launch_lookback_selftest(const uint32_t* keys, const uint32_t* vals, uint32_t* keys_out,
                                     uint32_t* vals_out, int64_t n, uint32_t first_ticket, int spin_limit, char* ws,
                                     uint32_t** err_out, cudaStream_t st);

cudaError_t launch_render_fwd(const sdgs_projected& p, const sdgs_bins& b, const sdgs_view& v,
                              float* image, float* final_T, uint32_t* n_contrib,
                              uint64_t* n_evaluated, cudaStream_t st);

size_t bwd_workspace_bytes(int64_t n);
int64_t alu_probe_sink_len();
cudaError_t launch_alu_probe(int kind, int iters, float* sink, double* ops, cudaStream_t st);
cudaError_t launch_densify(const sdgs_scene& s, const sdgs_view& v, const sdgs_densify_cfg& cfg,
                           const sdgs_densify& out, cudaStream_t st);
size_t agr_bwd_workspace_bytes(int64_t n);
cudaError_t launch_agr_refine(const sdgs_scene& s, const sdgs_agr& a, float t, float* mean7_out, float* L28_out,
                              cudaStream_t st);
cudaError_t launch_agr_refine_bwd(const sdgs_scene& s, const sdgs_agr& a, float t, const float* dmean7_hat,
                                  const float* dL28_hat, float* dmean7, float* dL28, const sdgs_agr_grads& g,
                                  char* ws, cudaStream_t st);
cudaError_t launch_render_bwd(const sdgs_scene& s, const sdgs_view& v, const sdgs_projected& p,
                              const sdgs_bins& b, const float* final_T, const uint32_t* n_contrib,
                              const float* dL_dimage, char* ws, const sdgs_grads& g,
                              cudaStream_t st);

}  // namespace sdgs
