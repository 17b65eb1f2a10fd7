// C-ABI entry points of libsdgs: argument validation, error reporting and dispatch to the
// kernel launchers.  Declarations and contracts are in include/sdgs.h.
#include <stdarg.h>
#include <stdio.h>

#include <cmath>
#include <mutex>

#include "common.cuh"

namespace sdgs {

static thread_local char g_error[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_error, sizeof(g_error), fmt, ap);
  va_end(ap);
}

int device_sm_count() {
  constexpr int kMaxDev = 64;
  static std::mutex mu;
  static int counts[kMaxDev] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return 152;
  std::lock_guard<std::mutex> lock(mu);
  if (counts[dev] == 0) {
    int c = 0;
    if (cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || c <= 0) c = 152;
    counts[dev] = c;
  }
  return counts[dev];
}

int cuda_status(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return SDGS_OK;
  set_error("%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
  return SDGS_ERR_CUDA;
}

static bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

static int check_scene(const sdgs_scene* s) {
  if (s == nullptr) { set_error("scene is NULL"); return SDGS_ERR_INVALID_ARG; }
  if (s->n < 0 || s->n >= (int64_t(1) << 31)) {
    set_error("scene n = %lld out of range [0, 2^31)", (long long)s->n);
    return SDGS_ERR_INVALID_ARG;
  }
  if (s->sh_degree != 3) { set_error("sh_degree must be 3 (got %d)", s->sh_degree); return SDGS_ERR_INVALID_ARG; }
  if (s->dir_mode != 0 && s->dir_mode != 1) { set_error("dir_mode must be 0 or 1 (got %d)", s->dir_mode); return SDGS_ERR_INVALID_ARG; }
  if (!(s->lambda_t >= 0.f) || !(s->lambda_d >= 0.f) || !std::isfinite(s->lambda_t) ||
      !std::isfinite(s->lambda_d)) {
    set_error("lambda_t / lambda_d must be finite and >= 0");
    return SDGS_ERR_INVALID_ARG;
  }
  if (s->n > 0) {
    if (!s->mean7 || !s->L28 || !s->opacity || !s->sh) { set_error("scene array is NULL"); return SDGS_ERR_INVALID_ARG; }
    if (!aligned(s->L28, 16) || !aligned(s->sh, 16) || !aligned(s->mean7, 4) || !aligned(s->opacity, 4)) {
      set_error("scene arrays must be aligned (L28 and sh to 16 bytes)");
      return SDGS_ERR_INVALID_ARG;
    }
  }
  return SDGS_OK;
}

static int check_view(const sdgs_view* v) {
  if (v == nullptr) { set_error("view is NULL"); return SDGS_ERR_INVALID_ARG; }
  if (v->width <= 0 || v->height <= 0 || v->width > 65535 * kTile || v->height > 65535 * kTile) {
    set_error("image size %d x %d out of range", v->width, v->height);
    return SDGS_ERR_INVALID_ARG;
  }
  if ((int64_t)((v->width + kTile - 1) / kTile) * ((v->height + kTile - 1) / kTile) > ((int64_t)1 << 26)) {
    set_error("image of %d x %d pixels has more than 2^26 tiles", v->width, v->height);
    return SDGS_ERR_INVALID_ARG;
  }
  if (!(v->fx > 0.f) || !(v->fy > 0.f) || !std::isfinite(v->fx) || !std::isfinite(v->fy) ||
      !std::isfinite(v->cx) || !std::isfinite(v->cy) || !(v->near_plane >= 0.f)) {
    set_error("bad intrinsics or near plane");
    return SDGS_ERR_INVALID_ARG;
  }
  for (int k = 0; k < 16; ++k)
    if (!std::isfinite(v->viewmat[k])) { set_error("viewmat is not finite"); return SDGS_ERR_INVALID_ARG; }
  if (!std::isfinite(v->t) || !std::isfinite(v->d[0]) || !std::isfinite(v->d[1]) || !std::isfinite(v->d[2])) {
    set_error("query t / d is not finite");
    return SDGS_ERR_INVALID_ARG;
  }
  return SDGS_OK;
}

static int check_projected(const sdgs_projected* p) {
  if (p == nullptr) { set_error("projected is NULL"); return SDGS_ERR_INVALID_ARG; }
  if (p->n < 0 || p->n >= (int64_t(1) << 30)) { set_error("projected n out of range [0, 2^30)"); return SDGS_ERR_INVALID_ARG; }
  if (p->n > 0) {
    if (!p->mean2d || !p->conic_opacity || !p->rgb || !p->depth || !p->rect || !p->radius) {
      set_error("projected array is NULL");
      return SDGS_ERR_INVALID_ARG;
    }
    if (!aligned(p->mean2d, 8) || !aligned(p->conic_opacity, 16) || !aligned(p->rect, 8) ||
        !aligned(p->rgb, 4) || !aligned(p->depth, 4) || !aligned(p->radius, 4)) {
      set_error("projected arrays misaligned (mean2d 8, conic_opacity 16, rect 8 bytes)");
      return SDGS_ERR_INVALID_ARG;
    }
  }
  return SDGS_OK;
}

static int check_bins(const sdgs_bins* b) {
  if (b == nullptr) { set_error("bins is NULL"); return SDGS_ERR_INVALID_ARG; }
  if (b->capacity < 0 || b->capacity >= (int64_t(1) << 30)) { set_error("bins capacity out of range [0, 2^30)"); return SDGS_ERR_INVALID_ARG; }
  if (!b->ranges || !b->num_instances || (b->capacity > 0 && !b->point_list)) {
    set_error("bins array is NULL");
    return SDGS_ERR_INVALID_ARG;
  }
  if (!aligned(b->ranges, 8) || !aligned(b->num_instances, 8)) { set_error("bins arrays misaligned"); return SDGS_ERR_INVALID_ARG; }
  return SDGS_OK;
}

}  // namespace sdgs

using namespace sdgs;

#define SDGS_TRY(x)                 \
  do {                              \
    const int _rc = (x);            \
    if (_rc != SDGS_OK) return _rc; \
  } while (0)

extern "C" {

const char* sdgs_version(void) { return "sdgs 0.1.0 sm_103a"; }

const char* sdgs_last_error(void) { return g_error; }

int sdgs_slice_project(const sdgs_scene* scene, const sdgs_view* view, const sdgs_projected* out,
                       void* stream) {
  g_error[0] = 0;
  SDGS_TRY(check_scene(scene));
  SDGS_TRY(check_view(view));
  SDGS_TRY(check_projected(out));
  if (out->n != scene->n) { set_error("projected n (%lld) != scene n (%lld)", (long long)out->n, (long long)scene->n); return SDGS_ERR_INVALID_ARG; }
  return cuda_status(launch_slice_project(*scene, *view, *out, (cudaStream_t)stream), "slice_project launch");
}

int sdgs_bin_workspace_size(int64_t n, int64_t capacity, int32_t width, int32_t height, size_t* bytes) {
  g_error[0] = 0;
  if (bytes == nullptr || n < 0 || n >= (int64_t(1) << 30) || capacity < 0 || capacity >= (int64_t(1) << 30) ||
      width <= 0 || height <= 0 || width > 65535 * kTile || height > 65535 * kTile ||
      (int64_t)((width + kTile - 1) / kTile) * ((height + kTile - 1) / kTile) > ((int64_t)1 << 26)) {
    set_error("bad arguments to sdgs_bin_workspace_size");
    return SDGS_ERR_INVALID_ARG;
  }
  *bytes = plan_bins(n, capacity, width, height).total;
  return SDGS_OK;
}

}  // extern "C"

// With a host count requested: synchronise, then report a sort that gave up waiting (never
// expected: every wait is on a block that is already running) or an overflow.  A sort that gave
// up leaves every tile range empty and the device instance count at -1.
static int finish_bin_sort(const BinPlan& plan, const char* ws, const sdgs_bins* out, int64_t* num_instances_host,
                           cudaStream_t st) {
  if (num_instances_host == nullptr) return SDGS_OK;
  uint32_t err = 0;
  SDGS_TRY(cuda_status(cudaMemcpyAsync(num_instances_host, out->num_instances, sizeof(int64_t),
                                       cudaMemcpyDeviceToHost, st), "copy instance count"));
  SDGS_TRY(cuda_status(cudaMemcpyAsync(&err, ws + plan.off_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st),
                       "copy sort status"));
  SDGS_TRY(cuda_status(cudaStreamSynchronize(st), "bin_sort synchronize"));
  if (err != 0 || *num_instances_host < 0) {
    set_error("binning sort: a look-back wait gave up (status 0x%x); every tile list was left empty", err);
    return SDGS_ERR_TIMEOUT;
  }
  if (*num_instances_host > out->capacity) {
    set_error("%lld instances exceed capacity %lld", (long long)*num_instances_host, (long long)out->capacity);
    return SDGS_ERR_OVERFLOW;
  }
  return SDGS_OK;
}

extern "C" {

static int bin_sort_impl(const sdgs_projected* proj, const sdgs_view* view, void* workspace,
                         size_t workspace_bytes, const sdgs_bins* out, int64_t* num_instances_host,
                         void* stream, uint32_t inject_err, uint32_t walk_ticket = 0, int spin_limit = 0) {
  g_error[0] = 0;
  SDGS_TRY(check_projected(proj));
  SDGS_TRY(check_view(view));
  SDGS_TRY(check_bins(out));
  const BinPlan plan = plan_bins(proj->n, out->capacity, view->width, view->height);
  if (workspace == nullptr || workspace_bytes < plan.total || !aligned(workspace, 256)) {
    set_error("workspace needs %zu bytes, 256-byte aligned (got %zu)", plan.total, workspace_bytes);
    return SDGS_ERR_WORKSPACE;
  }
  cudaStream_t st = (cudaStream_t)stream;
  if (walk_ticket != 0u && !plan.spans) {
    set_error("the span walk self-test needs an image of at most 256 tiles per side (span binning)");
    return SDGS_ERR_INVALID_ARG;
  }
  SDGS_TRY(cuda_status(launch_bin_sort(*proj, *view, plan, (char*)workspace, *out, st, inject_err, walk_ticket,
                                       spin_limit),
                       "bin_sort launch"));
  return finish_bin_sort(plan, (const char*)workspace, out, num_instances_host, st);
}

int sdgs_bin_sort(const sdgs_projected* proj, const sdgs_view* view, void* workspace,
                  size_t workspace_bytes, const sdgs_bins* out, int64_t* num_instances_host,
                  void* stream) {
  return bin_sort_impl(proj, view, workspace, workspace_bytes, out, num_instances_host, stream, 0u);
}

int sdgs_bin_sort_batch(const sdgs_projected* projs, const sdgs_view* views, void* const* workspaces,
                        const size_t* workspace_bytes, const sdgs_bins* outs, int32_t count,
                        int64_t* num_instances_host, void* stream) {
  g_error[0] = 0;
  if (count < 1 || count > kMaxBinBatch || !projs || !views || !workspaces || !workspace_bytes || !outs) {
    set_error("bin_sort_batch: count must be in [1, %d] and the arrays non-NULL", kMaxBinBatch);
    return SDGS_ERR_INVALID_ARG;
  }
  BinRequest reqs[kMaxBinBatch];
  for (int j = 0; j < count; ++j) {
    SDGS_TRY(check_projected(&projs[j]));
    SDGS_TRY(check_view(&views[j]));
    SDGS_TRY(check_bins(&outs[j]));
    const BinPlan plan = plan_bins(projs[j].n, outs[j].capacity, views[j].width, views[j].height);
    if (workspaces[j] == nullptr || workspace_bytes[j] < plan.total || !aligned(workspaces[j], 256)) {
      set_error("bin_sort_batch: workspace %d needs %zu bytes, 256-byte aligned (got %zu)", j, plan.total,
                workspace_bytes[j]);
      return SDGS_ERR_WORKSPACE;
    }
    reqs[j] = BinRequest{projs[j], views[j], plan, (char*)workspaces[j], outs[j], 0u};
  }
  cudaStream_t st = (cudaStream_t)stream;
  SDGS_TRY(cuda_status(launch_bin_sort_batch(reqs, count, st), "bin_sort_batch launch"));
  if (num_instances_host == nullptr) return SDGS_OK;
  int rc = SDGS_OK;
  for (int j = 0; j < count; ++j) {  // (the first synchronises; the rest are complete)
    const int r = finish_bin_sort(reqs[j].plan, reqs[j].ws, &outs[j], num_instances_host + j, st);
    if (r != SDGS_OK && rc == SDGS_OK) rc = r;
  }
  return rc;
}

int sdgs_bin_sort_failure_selftest(const sdgs_projected* proj, const sdgs_view* view, void* workspace,
                                   size_t workspace_bytes, const sdgs_bins* out, int64_t* num_instances_host,
                                   void* stream) {
  return bin_sort_impl(proj, view, workspace, workspace_bytes, out, num_instances_host, stream, 1u);
}

int sdgs_span_walk_selftest(const sdgs_projected* proj, const sdgs_view* view, void* workspace,
                            size_t workspace_bytes, const sdgs_bins* out, int64_t* num_instances_host,
                            uint32_t first_ticket, int32_t spin_limit, void* stream) {
  g_error[0] = 0;
  if (first_ticket > (1u << 20) || spin_limit < 1 || spin_limit > (1 << 20)) {
    set_error("span walk self-test: first_ticket must be <= 2^20 and spin_limit in [1, 2^20]");
    return SDGS_ERR_INVALID_ARG;
  }
  return bin_sort_impl(proj, view, workspace, workspace_bytes, out, num_instances_host, stream, 0u, first_ticket,
                       spin_limit);
}

}  // extern "C"

// ------------------------------------------------------------------------------------------
// Binning without a caller-provided workspace (sdgs_bin_sort_static).  Its scratch space is
// this file-scope device array.  In host code `g_bin_scratch` only names a host-side stand-in,
// so the kernels get the device address from cudaGetSymbolAddress, looked up once per device.
// Every byte of the workspace that binning reads is written earlier in the same call, so the
// array never needs clearing between calls.
// ------------------------------------------------------------------------------------------
static __device__ __align__(256) unsigned char g_bin_scratch[SDGS_STATIC_BIN_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

// The array's device address for the current device, looked up at the first call on that device
// and cached.  The cache is not invalidated by cudaDeviceReset: a caller that resets a device and
// keeps using the library in the same process must not call sdgs_bin_sort_static again.
int static_scratch(void** ptr) {
  int dev = 0;
  SDGS_TRY(cuda_status(cudaGetDevice(&dev), "cudaGetDevice"));
  if (dev < 0 || dev >= kMaxDevices) { set_error("device ordinal %d out of range", dev); return SDGS_ERR_INVALID_ARG; }
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (g_scratch_ptr[dev] == nullptr) {
    void* p = nullptr;
    SDGS_TRY(cuda_status(cudaGetSymbolAddress(&p, g_bin_scratch), "cudaGetSymbolAddress(bin scratch)"));
    g_scratch_ptr[dev] = p;
  }
  *ptr = g_scratch_ptr[dev];
  return SDGS_OK;
}
}  // namespace

extern "C" {

int sdgs_bin_sort_static(const sdgs_projected* proj, const sdgs_view* view, const sdgs_bins* out,
                         int64_t* num_instances_host, void* stream) {
  g_error[0] = 0;
  SDGS_TRY(check_projected(proj));
  SDGS_TRY(check_view(view));
  SDGS_TRY(check_bins(out));
  const BinPlan plan = plan_bins(proj->n, out->capacity, view->width, view->height);
  if (plan.total > SDGS_STATIC_BIN_SCRATCH_BYTES) {
    set_error("binning %lld Gaussians into %d tiles needs %zu bytes of scratch; the built-in scratch "
              "holds %zu (use sdgs_bin_sort with a workspace)",
              (long long)proj->n, plan.num_tiles, plan.total, (size_t)SDGS_STATIC_BIN_SCRATCH_BYTES);
    return SDGS_ERR_WORKSPACE;
  }
  void* ws = nullptr;
  SDGS_TRY(static_scratch(&ws));
  cudaStream_t st = (cudaStream_t)stream;
  SDGS_TRY(cuda_status(launch_bin_sort(*proj, *view, plan, (char*)ws, *out, st), "bin_sort launch"));
  return finish_bin_sort(plan, (const char*)ws, out, num_instances_host, st);
}

int sdgs_alu_peak_probe(int32_t kind, int32_t iters, float* sink, int64_t sink_len, double* ops, void* stream) {
  g_error[0] = 0;
  const int64_t need = alu_probe_sink_len();
  if (kind < 0 || kind > 2 || iters < 1 || ops == nullptr) {
    set_error("alu_peak_probe: kind in {0, 1, 2}, iters >= 1, ops not NULL");
    return SDGS_ERR_INVALID_ARG;
  }
  if (sink == nullptr || sink_len < need || !aligned(sink, 4)) {
    set_error("alu_peak_probe: sink needs %lld floats", (long long)need);
    return SDGS_ERR_WORKSPACE;
  }
  return cuda_status(launch_alu_probe(kind, iters, sink, ops, (cudaStream_t)stream), "alu probe launch");
}

int sdgs_lookback_selftest_workspace_size(int64_t n, size_t* bytes) {
  g_error[0] = 0;
  if (bytes == nullptr || n < 0 || n >= (int64_t(1) << 30)) {
    set_error("bad arguments to sdgs_lookback_selftest_workspace_size");
    return SDGS_ERR_INVALID_ARG;
  }
  *bytes = lookback_selftest_bytes(n);
  return SDGS_OK;
}

int sdgs_lookback_selftest(const uint32_t* keys, const uint32_t* vals, uint32_t* keys_out, uint32_t* vals_out,
                           int64_t n, uint32_t first_ticket, int32_t spin_limit, void* workspace,
                           size_t workspace_bytes, void* stream) {
  g_error[0] = 0;
  if (n < 0 || n >= (int64_t(1) << 30) || first_ticket > (1u << 20) || spin_limit < 1 || spin_limit > (1 << 20)) {
    set_error("lookback selftest: n in [0, 2^30), first_ticket <= 2^20, spin_limit in [1, 2^20]");
    return SDGS_ERR_INVALID_ARG;
  }
  if (n > 0 && (!keys || !vals || !keys_out || !vals_out)) { set_error("NULL key / value array"); return SDGS_ERR_INVALID_ARG; }
  const size_t need = lookback_selftest_bytes(n);
  if (workspace == nullptr || workspace_bytes < need || !aligned(workspace, 256)) {
    set_error("lookback selftest workspace needs %zu bytes, 256-byte aligned", need);
    return SDGS_ERR_WORKSPACE;
  }
  cudaStream_t st = (cudaStream_t)stream;
  uint32_t* err_dev = nullptr;
  SDGS_TRY(cuda_status(launch_lookback_selftest(keys, vals, keys_out, vals_out, n, first_ticket, spin_limit,
                                                (char*)workspace, &err_dev, st),
                       "lookback selftest launch"));
  uint32_t err = 0;
  SDGS_TRY(cuda_status(cudaMemcpyAsync(&err, err_dev, sizeof(uint32_t), cudaMemcpyDeviceToHost, st),
                       "copy sort status"));
  SDGS_TRY(cuda_status(cudaStreamSynchronize(st), "lookback selftest synchronize"));
  if (err != 0) {
    set_error("radix pass: a look-back wait gave up after %d rounds (status 0x%x)", spin_limit, err);
    return SDGS_ERR_TIMEOUT;
  }
  return SDGS_OK;
}

int sdgs_render_fwd(const sdgs_projected* proj, const sdgs_bins* bins, const sdgs_view* view,
                    float* image, float* final_T, uint32_t* n_contrib, uint64_t* n_evaluated,
                    void* stream) {
  g_error[0] = 0;
  SDGS_TRY(check_projected(proj));
  SDGS_TRY(check_bins(bins));
  SDGS_TRY(check_view(view));
  if (!image || !final_T || !n_contrib) { set_error("output image / final_T / n_contrib is NULL"); return SDGS_ERR_INVALID_ARG; }
  if (n_evaluated != nullptr && !aligned(n_evaluated, 8)) { set_error("n_evaluated misaligned"); return SDGS_ERR_INVALID_ARG; }
  return cuda_status(launch_render_fwd(*proj, *bins, *view, image, final_T, n_contrib, n_evaluated,
                                       (cudaStream_t)stream),
                     "render_fwd launch");
}

int sdgs_densify_stats(const sdgs_scene* scene, const sdgs_view* view, const sdgs_densify_cfg* cfg,
                       const sdgs_densify* out, void* stream) {
  g_error[0] = 0;
  SDGS_TRY(check_scene(scene));
  SDGS_TRY(check_view(view));
  if (cfg == nullptr || out == nullptr) { set_error("densify cfg / outputs are NULL"); return SDGS_ERR_INVALID_ARG; }
  if (!std::isfinite(cfg->extent) || !std::isfinite(cfg->split_pt) || !std::isfinite(cfg->split_t) ||
      !std::isfinite(cfg->prune_alpha)) {
    set_error("densify thresholds must be finite");
    return SDGS_ERR_INVALID_ARG;
  }
  if ((out->scale && !aligned(out->scale, 4)) || (out->rot && !aligned(out->rot, 4)) ||
      (out->pt_norm && !aligned(out->pt_norm, 4)) || (out->t_scale && !aligned(out->t_scale, 4))) {
    set_error("densify outputs misaligned");
    return SDGS_ERR_INVALID_ARG;
  }
  return cuda_status(launch_densify(*scene, *view, *cfg, *out, (cudaStream_t)stream), "densify launch");
}

static int check_agr(const sdgs_agr* a) {
  if (a == nullptr || !a->w1 || !a->b1 || !a->w2 || !a->b2) { set_error("AGR weights are NULL"); return SDGS_ERR_INVALID_ARG; }
  if (!aligned(a->w1, 4) || !aligned(a->b1, 4) || !aligned(a->w2, 4) || !aligned(a->b2, 4)) {
    set_error("AGR weights misaligned");
    return SDGS_ERR_INVALID_ARG;
  }
  return SDGS_OK;
}

int sdgs_agr_refine(const sdgs_scene* scene, const sdgs_agr* agr, float t, float* mean7_out, float* L28_out,
                    void* stream) {
  g_error[0] = 0;
  SDGS_TRY(check_scene(scene));
  SDGS_TRY(check_agr(agr));
  if (!std::isfinite(t)) { set_error("t is not finite"); return SDGS_ERR_INVALID_ARG; }
  if (scene->n > 0 && (!mean7_out || !L28_out || !aligned(mean7_out, 4) || !aligned(L28_out, 16))) {
    set_error("refined outputs NULL or misaligned (L28_out to 16 bytes)");
    return SDGS_ERR_INVALID_ARG;
  }
  if (scene->n > 0 && ((const float*)mean7_out == scene->mean7 || (const float*)L28_out == scene->L28)) {
    set_error("refined outputs alias the scene");
    return SDGS_ERR_INVALID_ARG;
  }
  return cuda_status(launch_agr_refine(*scene, *agr, t, mean7_out, L28_out, (cudaStream_t)stream), "agr launch");
}

int sdgs_agr_bwd_workspace_size(int64_t n, size_t* bytes) {
  if (bytes == nullptr || n < 0 || n >= (int64_t(1) << 31)) { set_error("bad arguments to sdgs_agr_bwd_workspace_size"); return SDGS_ERR_INVALID_ARG; }
  *bytes = agr_bwd_workspace_bytes(n);
  return SDGS_OK;
}

int sdgs_agr_refine_bwd(const sdgs_scene* scene, const sdgs_agr* agr, float t, const float* dmean7_hat,
                        const float* dL28_hat, float* dmean7, float* dL28, const sdgs_agr_grads* dagr,
                        void* workspace, size_t workspace_bytes, void* stream) {
  g_error[0] = 0;
  SDGS_TRY(check_scene(scene));
  SDGS_TRY(check_agr(agr));
  if (!std::isfinite(t)) { set_error("t is not finite"); return SDGS_ERR_INVALID_ARG; }
  if (dagr == nullptr || !dagr->dw1 || !dagr->db1 || !dagr->dw2 || !dagr->db2) {
    set_error("AGR gradient pointers are NULL");
    return SDGS_ERR_INVALID_ARG;
  }
  if (scene->n > 0 && (!dmean7_hat || !dL28_hat || !dmean7)) {
    set_error("AGR backward input / output pointer is NULL");
    return SDGS_ERR_INVALID_ARG;
  }
  const size_t need = agr_bwd_workspace_bytes(scene->n);
  if (workspace == nullptr || workspace_bytes < need || !aligned(workspace, 256)) {
    set_error("AGR backward workspace needs %zu bytes, 256-byte aligned", need);
    return SDGS_ERR_WORKSPACE;
  }
  return cuda_status(launch_agr_refine_bwd(*scene, *agr, t, dmean7_hat, dL28_hat, dmean7, dL28, *dagr,
                                           (char*)workspace, (cudaStream_t)stream),
                     "agr backward launch");
}

int sdgs_bwd_workspace_size(int64_t n, size_t* bytes) {
  g_error[0] = 0;
  if (bytes == nullptr || n < 0 || n >= (int64_t(1) << 31)) { set_error("bad arguments to sdgs_bwd_workspace_size"); return SDGS_ERR_INVALID_ARG; }
  *bytes = bwd_workspace_bytes(n);
  return SDGS_OK;
}

int sdgs_render_bwd(const sdgs_scene* scene, const sdgs_view* view, const sdgs_projected* proj,
                    const sdgs_bins* bins, const float* final_T, const uint32_t* n_contrib,
                    const float* dL_dimage, void* workspace, size_t workspace_bytes,
                    const sdgs_grads* grads, void* stream) {
  g_error[0] = 0;
  SDGS_TRY(check_scene(scene));
  SDGS_TRY(check_view(view));
  SDGS_TRY(check_projected(proj));
  SDGS_TRY(check_bins(bins));
  if (proj->n != scene->n) { set_error("projected n != scene n"); return SDGS_ERR_INVALID_ARG; }
  if (!final_T || !n_contrib || !dL_dimage || !grads || !grads->dmean7 || !grads->dL28 ||
      !grads->dopacity || !grads->dsh) {
    set_error("backward input or gradient pointer is NULL");
    return SDGS_ERR_INVALID_ARG;
  }
  if (grads->dlambda != nullptr && !aligned(grads->dlambda, 4)) { set_error("dlambda misaligned"); return SDGS_ERR_INVALID_ARG; }
  if (!aligned(grads->dL28, 16) || !aligned(grads->dsh, 16) || !aligned(grads->dmean7, 4) || !aligned(grads->dopacity, 4)) {
    set_error("gradient arrays misaligned (dL28 and dsh to 16 bytes)");
    return SDGS_ERR_INVALID_ARG;
  }
  const size_t need = bwd_workspace_bytes(scene->n);
  if (workspace == nullptr || workspace_bytes < need || !aligned(workspace, 256)) {
    set_error("backward workspace needs %zu bytes, 256-byte aligned", need);
    return SDGS_ERR_WORKSPACE;
  }
  return cuda_status(launch_render_bwd(*scene, *view, *proj, *bins, final_T, n_contrib, dL_dimage,
                                       (char*)workspace, *grads, (cudaStream_t)stream),
                     "render_bwd launch");
}

}  // extern "C"
