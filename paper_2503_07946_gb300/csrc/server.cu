// Render server over resident scenes (include/sdgs.h, sdgs_server_*).
//
// One worker thread owns all CUDA work of the server.  Requests wait in a FIFO queue; the worker
// admits the head of the queue whenever a slot (a stream plus its device buffers) is free and the
// device-memory budget covers the slot's buffers for that request.  Requests admitted in the same
// pass are sliced and projected by ONE batched launch on a batch stream (blockIdx.y = request);
// each request's binning, compositing and image copy then run on its own slot stream after an
// event from the batch stream, so the device overlaps several requests.  A host function at the
// end of each slot stream marks completion (and stamps the completion time).  If a request needs
// more (tile, Gaussian) instances than its bins hold, the worker grows them and re-runs binning
// and compositing for it.
#include <stdarg.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <memory>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"

namespace sdgs {

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t id = 0;
  int32_t scene = 0;
  sdgs_view view{};
  float* out = nullptr;
  Clock::time_point t_submit, t_done;
  int state = SDGS_REQ_QUEUED;
  int rc = SDGS_OK;
  int64_t capacity = 0;  // instance capacity of this request's bins
  int slot = -1;
};

struct Slot {
  cudaStream_t st = nullptr;
  Request* req = nullptr;
  // device buffers, grown on demand
  int64_t n_cap = 0;
  float *mean2d = nullptr, *conic_opacity = nullptr, *rgb = nullptr, *depth = nullptr;
  uint16_t* rect = nullptr;
  int32_t* radius = nullptr;
  int64_t k_cap = 0;
  uint32_t* point_list = nullptr;
  int tiles_cap = 0;
  uint32_t* ranges = nullptr;
  int64_t* num_instances = nullptr;
  size_t ws_cap = 0;
  void* ws = nullptr;
  int64_t pix_cap = 0;
  float* image = nullptr;
  float* final_T = nullptr;
  uint32_t* n_contrib = nullptr;
  int64_t* pinned_k = nullptr;
  size_t bytes = 0;
};

size_t proj_bytes(int64_t n) { return (size_t)n * (8 + 16 + 12 + 4 + 8 + 4); }
size_t pix_bytes(int64_t p) { return (size_t)p * (12 + 4 + 4); }

}  // namespace

}  // namespace sdgs

struct sdgs_server {
  sdgs_server_cfg cfg{};
  std::vector<sdgs_scene> scenes;
  std::vector<double> k_per_px;  // largest instances per pixel seen per scene
  std::deque<sdgs::Request*> queue;
  std::unordered_map<uint64_t, sdgs::Request*> requests;
  std::vector<sdgs::Slot> slots;
  // Written by the completion host functions without the mutex: a host function must never wait
  // on it, because the worker may hold it inside a CUDA call that waits for the streams.
  std::unique_ptr<std::atomic<int>[]> finished;        // per slot: 1 once the tail completed
  std::unique_ptr<std::atomic<int64_t>[]> finished_at;  // per slot: completion time (clock ticks)
  uint64_t next_id = 1;
  size_t bytes_allocated = 0;
  sdgs_server_stats stats{};
  uint64_t max_inflight = 0;
  bool stop = false;
  bool fatal = false;
  std::mutex mu;
  std::condition_variable work_cv;  // wakes the worker
  std::condition_variable done_cv;  // wakes waiters
  std::thread worker;
  // batched slicing
  cudaStream_t batch_stream = nullptr;
  cudaEvent_t batch_event = nullptr;
};

namespace sdgs {

namespace {

void host_done(void* arg);

struct DoneArg {
  sdgs_server* s;
  int slot;
};

// Largest instance capacity of a request: the binning sort's status words count in 30 bits.
constexpr int64_t kMaxCapacity = (int64_t(1) << 30) - 1;

int64_t capacity_estimate(const sdgs_server* s, int32_t scene, const sdgs_view& v) {
  const double px = (double)v.width * v.height;
  const double per = s->k_per_px[scene] > 0 ? s->k_per_px[scene] * 1.25 : 40.0;
  const double k = std::max(4096.0, per * px);
  return (int64_t)std::min(k, (double)kMaxCapacity);
}

size_t request_bytes(const sdgs_scene& sc, const sdgs_view& v, int64_t cap) {
  const BinPlan plan = plan_bins(sc.n, cap, v.width, v.height);
  const size_t tiles = (size_t)tiles_of(v.width) * tiles_of(v.height);
  return proj_bytes(sc.n) + (size_t)cap * 4 + tiles * 8 + 8 + plan.total + pix_bytes((int64_t)v.width * v.height);
}

// Free every buffer of a slot (the worker only calls this for idle slots).
void release_slot(sdgs_server* s, Slot& sl) {
  void* ptrs[] = {sl.mean2d, sl.conic_opacity, sl.rgb, sl.depth, sl.rect, sl.radius, sl.point_list,
                  sl.ranges, sl.num_instances, sl.ws, sl.image, sl.final_T, sl.n_contrib};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  s->bytes_allocated -= sl.bytes;
  sl.mean2d = sl.conic_opacity = sl.rgb = sl.depth = nullptr;
  sl.rect = nullptr;
  sl.radius = nullptr;
  sl.point_list = sl.ranges = nullptr;
  sl.num_instances = nullptr;
  sl.ws = nullptr;
  sl.image = sl.final_T = nullptr;
  sl.n_contrib = nullptr;
  sl.n_cap = sl.k_cap = sl.pix_cap = 0;
  sl.tiles_cap = 0;
  sl.ws_cap = 0;
  sl.bytes = 0;
}

template <typename T>
cudaError_t grow(T** p, size_t count) {
  if (*p) cudaFree(*p);
  *p = nullptr;
  return cudaMalloc(reinterpret_cast<void**>(p), std::max<size_t>(count, 1) * sizeof(T));
}

// Bytes the slot must add to hold this request.
size_t slot_growth(const Slot& sl, const sdgs_scene& sc, const sdgs_view& v, int64_t cap) {
  size_t g = 0;
  if (sl.n_cap < sc.n) g += proj_bytes(sc.n);
  if (sl.k_cap < cap) g += (size_t)cap * 4;
  const int tiles = tiles_of(v.width) * tiles_of(v.height);
  if (sl.tiles_cap < tiles) g += (size_t)tiles * 8 + 8;
  const size_t ws = plan_bins(sc.n, cap, v.width, v.height).total;
  if (sl.ws_cap < ws) g += ws;
  const int64_t px = (int64_t)v.width * v.height;
  if (sl.pix_cap < px) g += pix_bytes(px);
  return g;
}

// Make the slot's buffers big enough (reallocating the ones that are too small).
cudaError_t ensure_slot(sdgs_server* s, Slot& sl, const sdgs_scene& sc, const sdgs_view& v, int64_t cap) {
  cudaError_t e = cudaSuccess;
  const size_t before = sl.bytes;
  // a buffer that is too small is freed and re-allocated whole; the footprint follows the caps
  if (sl.n_cap < sc.n) {
    if ((e = grow(&sl.mean2d, 2 * sc.n)) || (e = grow(&sl.conic_opacity, 4 * sc.n)) ||
        (e = grow(&sl.rgb, 3 * sc.n)) || (e = grow(&sl.depth, sc.n)) || (e = grow(&sl.rect, 4 * sc.n)) ||
        (e = grow(&sl.radius, sc.n)))
      return e;
    sl.n_cap = sc.n;
  }
  if (sl.k_cap < cap) {
    if ((e = grow(&sl.point_list, cap))) return e;
    sl.k_cap = cap;
  }
  const int tiles = tiles_of(v.width) * tiles_of(v.height);
  if (sl.tiles_cap < tiles) {
    if ((e = grow(&sl.ranges, 2 * (size_t)tiles)) || (e = grow(&sl.num_instances, 1))) return e;
    sl.tiles_cap = tiles;
  }
  const size_t ws = plan_bins(sc.n, cap, v.width, v.height).total;
  if (sl.ws_cap < ws) {
    if (sl.ws) cudaFree(sl.ws);
    sl.ws = nullptr;
    if ((e = cudaMalloc(&sl.ws, ws))) return e;
    sl.ws_cap = ws;
  }
  const int64_t px = (int64_t)v.width * v.height;
  if (sl.pix_cap < px) {
    if ((e = grow(&sl.image, 3 * px)) || (e = grow(&sl.final_T, px)) || (e = grow(&sl.n_contrib, px))) return e;
    sl.pix_cap = px;
  }
  sl.bytes = proj_bytes(sl.n_cap) + (size_t)sl.k_cap * 4 + (size_t)sl.tiles_cap * 8 + 8 + sl.ws_cap +
             pix_bytes(sl.pix_cap);
  s->bytes_allocated += sl.bytes - before;
  return cudaSuccess;
}

sdgs_projected slot_projected(const Slot& sl, int64_t n) {
  sdgs_projected p;
  p.mean2d = sl.mean2d;
  p.conic_opacity = sl.conic_opacity;
  p.rgb = sl.rgb;
  p.depth = sl.depth;
  p.rect = sl.rect;
  p.radius = sl.radius;
  p.n = n;
  return p;
}

sdgs_bins slot_bins(const Slot& sl, int64_t cap) {
  sdgs_bins b;
  b.tile_keys = nullptr;
  b.point_list = sl.point_list;
  b.ranges = sl.ranges;
  b.num_instances = sl.num_instances;
  b.capacity = cap;
  return b;
}

// The binning arguments of a slot's request.
BinRequest slot_bin_request(const sdgs_server* s, const Slot& sl) {
  const Request* r = sl.req;
  const sdgs_scene& sc = s->scenes[r->scene];
  return BinRequest{slot_projected(sl, sc.n), r->view, plan_bins(sc.n, r->capacity, r->view.width, r->view.height),
                    (char*)sl.ws, slot_bins(sl, r->capacity), 0u};
}

// The instance count, compositing and the image copy on the slot's stream (after its binning),
// then the completion host function.
cudaError_t enqueue_render(sdgs_server* s, int slot_index) {
  Slot& sl = s->slots[slot_index];
  Request* r = sl.req;
  const sdgs_scene& sc = s->scenes[r->scene];
  const sdgs_projected p = slot_projected(sl, sc.n);
  const sdgs_bins b = slot_bins(sl, r->capacity);
  cudaError_t e;
  if ((e = cudaMemcpyAsync(sl.pinned_k, sl.num_instances, sizeof(int64_t), cudaMemcpyDeviceToHost, sl.st)))
    return e;
  if ((e = launch_render_fwd(p, b, r->view, sl.image, sl.final_T, sl.n_contrib, nullptr, sl.st))) return e;
  const size_t img = (size_t)r->view.width * r->view.height * 3 * sizeof(float);
  if ((e = cudaMemcpyAsync(r->out, sl.image, img, cudaMemcpyDefault, sl.st))) return e;
  s->finished[slot_index].store(0);
  DoneArg* arg = new DoneArg{s, slot_index};
  e = cudaLaunchHostFunc(sl.st, host_done, arg);
  if (e != cudaSuccess) delete arg;
  return e;
}

// Binning of one request on its slot's stream, then its render (a retry after an overflow).
cudaError_t enqueue_tail(sdgs_server* s, int slot_index) {
  Slot& sl = s->slots[slot_index];
  const BinRequest br = slot_bin_request(s, sl);
  cudaError_t e = launch_bin_sort(br.proj, br.view, br.plan, br.ws, br.out, sl.st);
  return e != cudaSuccess ? e : enqueue_render(s, slot_index);
}

void host_done(void* p) {
  DoneArg* a = static_cast<DoneArg*>(p);
  a->s->finished_at[a->slot].store(Clock::now().time_since_epoch().count());
  a->s->finished[a->slot].store(1);
  a->s->work_cv.notify_one();
  delete a;
}

void fail_request(sdgs_server* s, Request* r, int rc) {
  r->state = SDGS_REQ_FAILED;
  r->rc = rc;
  r->t_done = Clock::now();
  s->stats.failed++;
}

// Handle finished slots: retry overflowed requests, complete the rest.  Called with mu held.
void reap(sdgs_server* s) {
  for (int i = 0; i < (int)s->slots.size(); ++i) {
    Slot& sl = s->slots[i];
    if (!sl.req || !s->finished[i].load()) continue;
    Request* r = sl.req;
    const int64_t k = *sl.pinned_k;
    const double px = (double)r->view.width * r->view.height;
    if (k >= 0) s->k_per_px[r->scene] = std::max(s->k_per_px[r->scene], (double)k / px);
    if (k < 0) {  // a bounded wait of the binning sort gave up: the image holds only the background
      set_error("request %llu: binning gave up waiting", (unsigned long long)r->id);
      fail_request(s, r, SDGS_ERR_TIMEOUT);
    } else if (k > kMaxCapacity) {
      set_error("request %llu: %lld instances exceed the largest capacity", (unsigned long long)r->id, (long long)k);
      fail_request(s, r, SDGS_ERR_OVERFLOW);
    } else if (k > r->capacity) {  // grow the instance lists and bin + composite again
      r->capacity = std::min<int64_t>((int64_t)(k * 1.1) + 4096, kMaxCapacity);
      s->stats.retried++;
      const size_t growth = slot_growth(sl, s->scenes[r->scene], r->view, r->capacity);
      if (s->bytes_allocated + growth <= s->cfg.hbm_budget_bytes) {
        cudaError_t e = ensure_slot(s, sl, s->scenes[r->scene], r->view, r->capacity);
        if (e == cudaSuccess) e = enqueue_tail(s, i);
        if (e == cudaSuccess) continue;
        set_error("server retry: %s", cudaGetErrorString(e));
        fail_request(s, r, SDGS_ERR_CUDA);
      } else {
        // the larger lists do not fit beside the other slots now: back to the head of the queue,
        // where admission waits for memory as it does for a new request
        r->state = SDGS_REQ_QUEUED;
        r->slot = -1;
        s->queue.push_front(r);
      }
    } else {
      r->state = SDGS_REQ_DONE;
      r->t_done = Clock::time_point(Clock::duration(s->finished_at[i].load()));
      s->stats.completed++;
    }
    sl.req = nullptr;
    s->finished[i].store(0);
    s->done_cv.notify_all();
  }
}

// Admit queued requests into free slots within the budget; slice them in one batched launch.
void admit(sdgs_server* s) {
  std::vector<int> started;
  while (!s->queue.empty()) {
    Request* r = s->queue.front();
    int free_slot = -1;
    for (int i = 0; i < (int)s->slots.size(); ++i)
      if (!s->slots[i].req) { free_slot = i; break; }
    if (free_slot < 0) break;
    const sdgs_scene& sc = s->scenes[r->scene];
    if (r->capacity == 0) r->capacity = capacity_estimate(s, r->scene, r->view);
    size_t growth = slot_growth(s->slots[free_slot], sc, r->view, r->capacity);
    if (s->bytes_allocated + growth > s->cfg.hbm_budget_bytes) {
      // release the buffers of other idle slots to make room
      for (int i = 0; i < (int)s->slots.size() && s->bytes_allocated + growth > s->cfg.hbm_budget_bytes; ++i)
        if (!s->slots[i].req && i != free_slot && s->slots[i].bytes) release_slot(s, s->slots[i]);
      if (s->bytes_allocated + growth > s->cfg.hbm_budget_bytes) {
        if (s->slots[free_slot].bytes) {  // shrink-to-fit this slot too before giving up
          release_slot(s, s->slots[free_slot]);
          growth = slot_growth(s->slots[free_slot], sc, r->view, r->capacity);
        }
        if (s->bytes_allocated + growth > s->cfg.hbm_budget_bytes) break;  // wait for memory
      }
    }
    s->queue.pop_front();
    Slot& sl = s->slots[free_slot];
    cudaError_t e = ensure_slot(s, sl, sc, r->view, r->capacity);
    if (e != cudaSuccess) {
      set_error("server allocation: %s", cudaGetErrorString(e));
      fail_request(s, r, SDGS_ERR_CUDA);
      s->done_cv.notify_all();
      continue;
    }
    sl.req = r;
    s->finished[free_slot].store(0);
    r->slot = free_slot;
    r->state = SDGS_REQ_RUNNING;
    started.push_back(free_slot);
  }
  if (started.empty()) return;
  uint64_t inflight = 0;
  for (auto& sl : s->slots) inflight += sl.req ? 1 : 0;
  s->max_inflight = std::max(s->max_inflight, inflight);
  // batched slicing of every request admitted in this pass (8 per launch, arguments by value)
  std::vector<SliceRequest> slices;
  for (size_t j = 0; j < started.size(); ++j) {
    Slot& sl = s->slots[started[j]];
    const sdgs_scene& sc = s->scenes[sl.req->scene];
    slices.push_back(SliceRequest{sc, sl.req->view, slot_projected(sl, sc.n)});
  }
  cudaError_t e = launch_slice_project_batch(slices.data(), (int)slices.size(), s->batch_stream);
  // binning of the same requests, kMaxBinBatch per launch sequence, on the batch stream
  for (size_t j0 = 0; j0 < started.size() && e == cudaSuccess; j0 += kMaxBinBatch) {
    BinRequest reqs[kMaxBinBatch];
    int count = 0;
    for (size_t j = j0; j < started.size() && count < kMaxBinBatch; ++j)
      reqs[count++] = slot_bin_request(s, s->slots[started[j]]);
    e = launch_bin_sort_batch(reqs, count, s->batch_stream);
  }
  if (e == cudaSuccess) e = cudaEventRecord(s->batch_event, s->batch_stream);
  s->stats.batches++;
  s->stats.max_batch = std::max<uint64_t>(s->stats.max_batch, started.size());
  for (int idx : started) {
    Slot& sl = s->slots[idx];
    cudaError_t e2 = e;
    if (e2 == cudaSuccess) e2 = cudaStreamWaitEvent(sl.st, s->batch_event, 0);
    if (e2 == cudaSuccess) e2 = enqueue_render(s, idx);
    if (e2 != cudaSuccess) {
      set_error("server launch: %s", cudaGetErrorString(e2));
      fail_request(s, sl.req, SDGS_ERR_CUDA);
      sl.req = nullptr;
      s->fatal = true;
      s->done_cv.notify_all();
    }
  }
}

void worker_main(sdgs_server* s) {
  cudaSetDevice(s->cfg.device);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    reap(s);
    bool busy = false;
    for (auto& sl : s->slots) busy |= sl.req != nullptr;
    if (s->stop && !busy) break;
    auto wait = std::chrono::microseconds(2000);
    if (!s->stop && !s->fatal && !s->queue.empty()) {
      // batching window: with free slots to spare, let the queue fill until the oldest request
      // has waited batch_window_us
      int free_slots = 0;
      for (auto& sl : s->slots) free_slots += sl.req == nullptr;
      const auto age = Clock::now() - s->queue.front()->t_submit;
      const auto window = std::chrono::microseconds(s->cfg.batch_window_us);
      if (s->cfg.batch_window_us > 0 && (int)s->queue.size() < free_slots && age < window) {
        wait = std::chrono::duration_cast<std::chrono::microseconds>(window - age) + std::chrono::microseconds(1);
      } else {
        admit(s);
      }
    }
    s->work_cv.wait_for(lk, wait);
  }
  // requests that never started
  for (Request* r : s->queue) fail_request(s, r, SDGS_ERR_BUSY);
  s->queue.clear();
  s->done_cv.notify_all();
}

int check_server_view(const sdgs_view* v) {
  if (!v || v->width <= 0 || v->height <= 0 || v->width > 65535 * kTile || v->height > 65535 * kTile ||
      (int64_t)((v->width + kTile - 1) / kTile) * ((v->height + kTile - 1) / kTile) > ((int64_t)1 << 26) ||
      !(v->fx > 0.f) || !(v->fy > 0.f)) {
    set_error("bad view");
    return SDGS_ERR_INVALID_ARG;
  }
  return SDGS_OK;
}

}  // namespace

}  // namespace sdgs

using namespace sdgs;

extern "C" {

int sdgs_server_create(const sdgs_server_cfg* cfg, sdgs_server** out) {
  if (!cfg || !out || cfg->max_slots < 1 || cfg->max_slots > 64 || cfg->queue_capacity < 1 ||
      cfg->hbm_budget_bytes == 0 || cfg->batch_window_us < 0 || cfg->batch_window_us > 1000000) {
    set_error("bad server configuration");
    return SDGS_ERR_INVALID_ARG;
  }
  *out = nullptr;
  sdgs_server* s = new sdgs_server();
  s->cfg = *cfg;
  int rc = SDGS_OK;
  if ((rc = cuda_status(cudaSetDevice(cfg->device), "cudaSetDevice"))) { delete s; return rc; }
  s->slots.resize(cfg->max_slots);
  s->finished.reset(new std::atomic<int>[cfg->max_slots]);
  s->finished_at.reset(new std::atomic<int64_t>[cfg->max_slots]);
  for (int i = 0; i < cfg->max_slots; ++i) {
    s->finished[i].store(0);
    s->finished_at[i].store(0);
  }
  cudaError_t e = cudaStreamCreateWithFlags(&s->batch_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->batch_event, cudaEventDisableTiming);
  for (auto& sl : s->slots) {
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&sl.pinned_k), sizeof(int64_t));
  }
  if (e != cudaSuccess) {
    rc = cuda_status(e, "server create");
    sdgs_server_destroy(s);
    return rc;
  }
  s->worker = std::thread(worker_main, s);
  *out = s;
  return SDGS_OK;
}

int sdgs_server_add_scene(sdgs_server* s, const sdgs_scene* sc, int32_t* scene_id) {
  if (!s || !sc || !scene_id || sc->n < 0 || sc->n >= (int64_t(1) << 31) || sc->sh_degree != 3 ||
      (sc->n > 0 && (!sc->mean7 || !sc->L28 || !sc->opacity || !sc->sh))) {
    set_error("bad scene");
    return SDGS_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  s->scenes.push_back(*sc);
  s->k_per_px.push_back(0.0);
  *scene_id = (int32_t)s->scenes.size() - 1;
  return SDGS_OK;
}

int sdgs_server_submit(sdgs_server* s, int32_t scene_id, const sdgs_view* view, float* out_image,
                       uint64_t* req_id) {
  if (!s || !req_id || !out_image) { set_error("NULL argument"); return SDGS_ERR_INVALID_ARG; }
  const int vrc = check_server_view(view);
  if (vrc != SDGS_OK) return vrc;
  std::lock_guard<std::mutex> lk(s->mu);
  if (scene_id < 0 || scene_id >= (int32_t)s->scenes.size()) { set_error("unknown scene %d", scene_id); return SDGS_ERR_NOT_FOUND; }
  if (s->stop || s->fatal) { set_error("server is stopping or failed"); return SDGS_ERR_BUSY; }
  if ((int)s->queue.size() >= s->cfg.queue_capacity) { set_error("queue full"); return SDGS_ERR_BUSY; }
  const int64_t cap = capacity_estimate(s, scene_id, *view);
  const size_t need = request_bytes(s->scenes[scene_id], *view, cap);
  if (need > s->cfg.hbm_budget_bytes) {
    set_error("request needs %zu bytes, budget is %zu", need, s->cfg.hbm_budget_bytes);
    return SDGS_ERR_OOM_BUDGET;
  }
  Request* r = new Request();
  r->id = s->next_id++;
  r->scene = scene_id;
  r->view = *view;
  r->out = out_image;
  r->t_submit = Clock::now();
  s->requests[r->id] = r;
  s->queue.push_back(r);
  s->stats.submitted++;
  *req_id = r->id;
  s->work_cv.notify_one();
  return SDGS_OK;
}

int sdgs_server_poll(sdgs_server* s, uint64_t req_id, int32_t* state, float* latency_ms) {
  if (!s) return SDGS_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->requests.find(req_id);
  if (it == s->requests.end()) { set_error("unknown request"); return SDGS_ERR_NOT_FOUND; }
  const Request* r = it->second;
  if (state) *state = r->state;
  if (latency_ms)
    *latency_ms = (r->state >= SDGS_REQ_DONE)
                      ? std::chrono::duration<float, std::milli>(r->t_done - r->t_submit).count()
                      : 0.f;
  return SDGS_OK;
}

int sdgs_server_wait(sdgs_server* s, uint64_t req_id, int32_t timeout_ms, float* latency_ms) {
  if (!s) return SDGS_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->requests.find(req_id);
  if (it == s->requests.end()) { set_error("unknown request"); return SDGS_ERR_NOT_FOUND; }
  Request* r = it->second;
  const bool ok = s->done_cv.wait_for(lk, std::chrono::milliseconds(std::max(0, timeout_ms)),
                                      [&] { return r->state >= SDGS_REQ_DONE; });
  if (!ok) { set_error("request %llu not finished", (unsigned long long)req_id); return SDGS_ERR_TIMEOUT; }
  if (latency_ms) *latency_ms = std::chrono::duration<float, std::milli>(r->t_done - r->t_submit).count();
  return r->state == SDGS_REQ_DONE ? SDGS_OK : r->rc;
}

int sdgs_server_release(sdgs_server* s, uint64_t req_id) {
  if (!s) return 0;
  std::lock_guard<std::mutex> lk(s->mu);
  int n = 0;
  for (auto it = s->requests.begin(); it != s->requests.end();) {
    if ((req_id == 0 || it->first == req_id) && it->second->state >= SDGS_REQ_DONE) {
      delete it->second;
      it = s->requests.erase(it);
      ++n;
    } else {
      ++it;
    }
  }
  return n;
}

int sdgs_server_get_stats(sdgs_server* s, sdgs_server_stats* out) {
  if (!s || !out) return SDGS_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->stats;
  out->max_inflight = s->max_inflight;
  out->bytes_allocated = s->bytes_allocated;
  return SDGS_OK;
}

void sdgs_server_destroy(sdgs_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->work_cv.notify_all();
  if (s->worker.joinable()) s->worker.join();
  cudaSetDevice(s->cfg.device);
  for (auto& sl : s->slots) {
    if (sl.st) cudaStreamSynchronize(sl.st);
    release_slot(s, sl);
    if (sl.st) cudaStreamDestroy(sl.st);
    if (sl.pinned_k) cudaFreeHost(sl.pinned_k);
  }
  if (s->batch_stream) {
    cudaStreamSynchronize(s->batch_stream);
    cudaStreamDestroy(s->batch_stream);
  }
  if (s->batch_event) cudaEventDestroy(s->batch_event);
  for (auto& kv : s->requests) delete kv.second;
  delete s;
}

}  // extern "C"
