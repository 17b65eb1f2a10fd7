// Tile binning: the stable sort of (tile << 32 | depth bits) instance keys, done as an LSD radix
// sort whose depth digits are sorted BEFORE the instances are duplicated.
//
// Every instance of one Gaussian carries the same depth, and duplication emits instances in the
// order of the Gaussians it is given.  So the low (depth) passes of an LSD sort over the K
// instances give the same order as sorting the n Gaussians by depth first (stable, id order for
// ties) and emitting their instances in that order.  Only the tile digits are then sorted over
// the K instances: ceil(log2(tiles) / 8) passes instead of ceil((log2(tiles) + 32) / 8).
//
// Each radix pass is reduce-then-scan with no inter-block waiting: an upsweep writes a per-block
// digit histogram (digit-major), a device-wide exclusive scan turns it into block offsets, and a
// downsweep ranks the block's keys stably (warp match + per-warp counters) and scatters them
// through shared memory so that runs of one digit are written contiguously.
#include "common.cuh"

namespace sdgs {

namespace {

constexpr int kRadixThreads = 256;
constexpr int kRadixItems = 16;
constexpr int kRadixTile = kRadixThreads * kRadixItems;  // keys per block
constexpr int kRadixWarps = kRadixThreads / 32;
constexpr int kBins = 256;

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanChunk = kScanThreads * kScanItems;

// Element count: static, or read from device memory (clipped to cap) so that the launch
// configuration does not depend on data.
__device__ __forceinline__ int64_t element_count(const int64_t* nptr, int64_t n_static, int64_t cap) {
  if (nptr == nullptr) return n_static;
  const int64_t k = *nptr;
  return k < cap ? k : cap;
}

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

template <typename T>
__device__ __forceinline__ T warp_inclusive_scan(T x) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

// Inclusive scan across the block (blockDim.x = NT, a multiple of 32); *total gets the block sum.
template <typename T, int NT>
__device__ __forceinline__ T block_inclusive_scan(T x, T* total) {
  __shared__ T s_warp[NT / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T incl = warp_inclusive_scan(x);
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    T w = lane < NT / 32 ? s_warp[lane] : T(0);
    w = warp_inclusive_scan(w);
    if (lane < NT / 32) s_warp[lane] = w;
  }
  __syncthreads();
  if (warp > 0) incl += s_warp[warp - 1];
  *total = s_warp[NT / 32 - 1];
  __syncthreads();
  return incl;
}

// ------------------------------------------------------------------------------------------
// Device-wide exclusive scan: reduce per chunk, scan the chunk sums in one block, scan chunks.
// ------------------------------------------------------------------------------------------

template <typename TIn, typename TOut>
__global__ void __launch_bounds__(kScanThreads) scan_reduce_kernel(const TIn* in, int64_t n,
                                                                    TOut* partials) {
  const int64_t base = (int64_t)blockIdx.x * kScanChunk;
  TOut sum = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const int64_t i = base + k * kScanThreads + threadIdx.x;
    if (i < n) sum += (TOut)in[i];
  }
  TOut total;
  block_inclusive_scan<TOut, kScanThreads>(sum, &total);
  if (threadIdx.x == 0) partials[blockIdx.x] = total;
}

template <typename T>
__global__ void __launch_bounds__(1024) scan_partials_kernel(T* partials, int64_t nb, int64_t* total_out) {
  T carry = 0;
  for (int64_t base = 0; base < nb; base += 1024) {
    const int64_t i = base + threadIdx.x;
    const T x = i < nb ? partials[i] : T(0);
    T tot;
    const T incl = block_inclusive_scan<T, 1024>(x, &tot);
    if (i < nb) partials[i] = carry + incl - x;
    carry += tot;
  }
  if (threadIdx.x == 0 && total_out != nullptr) *total_out = (int64_t)carry;
}

template <typename TIn, typename TOut>
__global__ void __launch_bounds__(kScanThreads) scan_down_kernel(const TIn* in, int64_t n,
                                                                  const TOut* partials, TOut* out) {
  __shared__ TOut s[kScanChunk];
  const int64_t base = (int64_t)blockIdx.x * kScanChunk;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const int j = k * kScanThreads + threadIdx.x;
    s[j] = (base + j < n) ? (TOut)in[base + j] : TOut(0);
  }
  __syncthreads();
  TOut v[kScanItems];
  TOut local = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = local;
    local += s[threadIdx.x * kScanItems + k];
  }
  TOut tot;
  const TOut incl = block_inclusive_scan<TOut, kScanThreads>(local, &tot);
  const TOut off = partials[blockIdx.x] + incl - local;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) s[threadIdx.x * kScanItems + k] = off + v[k];
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const int j = k * kScanThreads + threadIdx.x;
    if (base + j < n) out[base + j] = s[j];
  }
}

template <typename TIn, typename TOut>
cudaError_t exclusive_scan(const TIn* in, int64_t n, TOut* out, uint64_t* partials,
                           int64_t* total_out, cudaStream_t st) {
  const int64_t nb = (n + kScanChunk - 1) / kScanChunk;
  TOut* part = reinterpret_cast<TOut*>(partials);
  if (nb > 0) scan_reduce_kernel<TIn, TOut><<<(unsigned)nb, kScanThreads, 0, st>>>(in, n, part);
  scan_partials_kernel<TOut><<<1, 1024, 0, st>>>(part, nb, total_out);
  if (nb > 0) scan_down_kernel<TIn, TOut><<<(unsigned)nb, kScanThreads, 0, st>>>(in, n, part, out);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// Radix pass kernels (8-bit digit at `shift`).
// ------------------------------------------------------------------------------------------

__global__ void __launch_bounds__(kRadixThreads)
radix_upsweep_kernel(const uint32_t* __restrict__ keys, const int64_t* nptr, int64_t n_static,
                     int64_t cap, int shift, uint32_t* __restrict__ hist, int64_t nblocks) {
  __shared__ uint32_t s_hist[kRadixWarps][kBins];
  for (int i = threadIdx.x; i < kRadixWarps * kBins; i += kRadixThreads) (&s_hist[0][0])[i] = 0;
  __syncthreads();
  const int64_t n = element_count(nptr, n_static, cap);
  const int64_t base = (int64_t)blockIdx.x * kRadixTile;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (base < n) {
    const int64_t wbase = base + (int64_t)warp * 32 * kRadixItems;
#pragma unroll 4
    for (int r = 0; r < kRadixItems; ++r) {
      const int64_t idx = wbase + r * 32 + lane;
      const bool valid = idx < n;
      const uint32_t d = valid ? ((keys[idx] >> shift) & 0xffu) : 0x100u;
      const unsigned peers = __match_any_sync(0xffffffffu, d);
      if (valid && lane == __ffs(peers) - 1) s_hist[warp][d] += __popc(peers);
      __syncwarp();
    }
  }
  __syncthreads();
  uint32_t tot = 0;
#pragma unroll
  for (int w = 0; w < kRadixWarps; ++w) tot += s_hist[w][threadIdx.x];
  hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kRadixThreads)
radix_downsweep_kernel(const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
                       uint32_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out,
                       const int64_t* nptr, int64_t n_static, int64_t cap, int shift,
                       const uint32_t* __restrict__ hist, int64_t nblocks) {
  __shared__ uint32_t s_keys[kRadixTile];
  __shared__ uint32_t s_vals[kRadixTile];
  __shared__ uint32_t s_whist[kRadixWarps][kBins];
  __shared__ uint32_t s_dstart[kBins];
  __shared__ uint32_t s_gbase[kBins];
  const int64_t n = element_count(nptr, n_static, cap);
  const int64_t base = (int64_t)blockIdx.x * kRadixTile;
  if (base >= n) return;
  for (int i = threadIdx.x; i < kRadixWarps * kBins; i += kRadixThreads) (&s_whist[0][0])[i] = 0;
  __syncthreads();

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned lt = lanemask_lt();
  const int64_t wbase = base + (int64_t)warp * 32 * kRadixItems;
  uint32_t key[kRadixItems], val[kRadixItems], rank[kRadixItems];
#pragma unroll
  for (int r = 0; r < kRadixItems; ++r) {
    const int64_t idx = wbase + r * 32 + lane;
    const bool valid = idx < n;
    key[r] = valid ? keys_in[idx] : 0u;
    val[r] = valid ? vals_in[idx] : 0u;
  }
#pragma unroll
  for (int r = 0; r < kRadixItems; ++r) {
    const bool valid = wbase + r * 32 + lane < n;
    const uint32_t d = valid ? ((key[r] >> shift) & 0xffu) : 0x100u;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const uint32_t before = valid ? s_whist[warp][d] : 0u;
    __syncwarp();
    if (valid && lane == __ffs(peers) - 1) s_whist[warp][d] = before + __popc(peers);
    __syncwarp();
    rank[r] = before + __popc(peers & lt);
  }
  __syncthreads();
  {
    const int dg = threadIdx.x;
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < kRadixWarps; ++w) {
      const uint32_t c = s_whist[w][dg];
      s_whist[w][dg] = run;
      run += c;
    }
    uint32_t tot;
    const uint32_t incl = block_inclusive_scan<uint32_t, kRadixThreads>(run, &tot);
    s_dstart[dg] = incl - run;
    s_gbase[dg] = hist[(int64_t)dg * nblocks + blockIdx.x];
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kRadixItems; ++r) {
    if (wbase + r * 32 + lane < n) {
      const uint32_t d = (key[r] >> shift) & 0xffu;
      const uint32_t pos = s_dstart[d] + s_whist[warp][d] + rank[r];
      s_keys[pos] = key[r];
      s_vals[pos] = val[r];
    }
  }
  __syncthreads();
  const int cnt = (int)((n - base) < kRadixTile ? (n - base) : kRadixTile);
  for (int i = threadIdx.x; i < cnt; i += kRadixThreads) {
    const uint32_t k = s_keys[i];
    const uint32_t d = (k >> shift) & 0xffu;
    const uint32_t g = s_gbase[d] + (uint32_t)i - s_dstart[d];
    keys_out[g] = k;
    vals_out[g] = s_vals[i];
  }
}

// Sorts (keys, vals) by bits [0, bits) in passes of 8 bits, ping-ponging between buffers 0 and 1;
// returns the index of the buffer that holds the result.
int radix_sort(uint32_t* keys[2], uint32_t* vals[2], const int64_t* nptr, int64_t n_static,
               int64_t cap, int bits, uint32_t* hist, uint64_t* partials, cudaStream_t st) {
  const int64_t nblocks = (cap + kRadixTile - 1) / kRadixTile;
  int cur = 0;
  if (nblocks == 0) return cur;
  for (int shift = 0; shift < bits; shift += 8) {
    radix_upsweep_kernel<<<(unsigned)nblocks, kRadixThreads, 0, st>>>(keys[cur], nptr, n_static,
                                                                        cap, shift, hist, nblocks);
    exclusive_scan<uint32_t, uint32_t>(hist, (int64_t)kBins * nblocks, hist, partials, nullptr, st);
    radix_downsweep_kernel<<<(unsigned)nblocks, kRadixThreads, 0, st>>>(
        keys[cur], vals[cur], keys[cur ^ 1], vals[cur ^ 1], nptr, n_static, cap, shift, hist,
        nblocks);
    cur ^= 1;
  }
  return cur;
}

// ------------------------------------------------------------------------------------------
// Binning-specific kernels.
// ------------------------------------------------------------------------------------------

__global__ void depth_keys_kernel(const float* __restrict__ depth, const ushort4* __restrict__ rect,
                                  int64_t n, uint32_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const ushort4 r = rect[i];
  const bool vis = r.z > r.x && r.w > r.y;
  keys[i] = vis ? __float_as_uint(depth[i]) : 0xffffffffu;  // visible depths are positive
  vals[i] = (uint32_t)i;
}

// Rectangles are clipped to the tile grid here and in duplicate_kernel, so records that come
// from the caller rather than from slice_project can never address a tile outside the image.
__device__ __forceinline__ ushort4 clip_rect(ushort4 r, int tiles_x, int tiles_y) {
  r.x = (unsigned short)min((int)r.x, tiles_x);
  r.z = (unsigned short)min((int)r.z, tiles_x);
  r.y = (unsigned short)min((int)r.y, tiles_y);
  r.w = (unsigned short)min((int)r.w, tiles_y);
  return r;
}

__global__ void tile_counts_kernel(const uint32_t* __restrict__ order, const ushort4* __restrict__ rect,
                                   int64_t n, int tiles_x, int tiles_y, uint32_t* __restrict__ counts) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const ushort4 r = clip_rect(rect[order[s]], tiles_x, tiles_y);
  const int w = (int)r.z - (int)r.x, h = (int)r.w - (int)r.y;
  counts[s] = (w > 0 && h > 0) ? (uint32_t)(w * h) : 0u;
}

__global__ void duplicate_kernel(const uint32_t* __restrict__ order, const uint64_t* __restrict__ offsets,
                                 const ushort4* __restrict__ rect, int tiles_x, int tiles_y, int64_t n,
                                 int64_t cap, uint32_t* __restrict__ tile_keys, uint32_t* __restrict__ vals) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const uint32_t g = order[s];
  const ushort4 r = clip_rect(rect[g], tiles_x, tiles_y);
  if (!(r.z > r.x && r.w > r.y)) return;
  uint64_t off = offsets[s];
  for (int y = r.y; y < r.w; ++y) {
    for (int x = r.x; x < r.z; ++x) {
      if (off >= (uint64_t)cap) return;
      tile_keys[off] = (uint32_t)(y * tiles_x + x);
      vals[off] = g;
      ++off;
    }
  }
}

__global__ void ranges_kernel(const uint32_t* __restrict__ keys, const int64_t* nptr, int64_t cap,
                              uint2* __restrict__ ranges) {
  const int64_t n = element_count(nptr, 0, cap);
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const uint32_t t = keys[j];
  if (j == 0 || keys[j - 1] != t) ranges[t].x = (uint32_t)j;
  if (j == n - 1 || keys[j + 1] != t) ranges[t].y = (uint32_t)(j + 1);
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

BinPlan plan_bins(int64_t n, int64_t capacity, int width, int height) {
  BinPlan p;
  p.n = n;
  p.capacity = capacity;
  p.num_tiles = tiles_of(width) * tiles_of(height);
  int bits = 0;
  while ((1ll << bits) < p.num_tiles) ++bits;
  p.tile_bits = bits;
  const int64_t nb_d = (n + kRadixTile - 1) / kRadixTile;
  const int64_t nb_i = (capacity + kRadixTile - 1) / kRadixTile;
  p.hist_blocks = nb_d > nb_i ? nb_d : nb_i;
  const int64_t hist_entries = (int64_t)kBins * p.hist_blocks;
  const int64_t part_a = (hist_entries + kScanChunk - 1) / kScanChunk;
  const int64_t part_b = (n + kScanChunk - 1) / kScanChunk;
  p.partial_cap = (part_a > part_b ? part_a : part_b) + 1;
  size_t off = 0;
  for (int k = 0; k < 2; ++k) { p.off_dkeys[k] = off; off += align256(sizeof(uint32_t) * n); }
  for (int k = 0; k < 2; ++k) { p.off_dvals[k] = off; off += align256(sizeof(uint32_t) * n); }
  p.off_counts = off; off += align256(sizeof(uint64_t) * (n + 1));
  p.off_ikeys = off; off += align256(sizeof(uint32_t) * capacity);
  p.off_ivals = off; off += align256(sizeof(uint32_t) * capacity);
  p.off_hist = off; off += align256(sizeof(uint32_t) * hist_entries);
  p.off_partials = off; off += align256(sizeof(uint64_t) * p.partial_cap);
  p.off_scalars = off; off += align256(sizeof(uint64_t) * 8);
  p.total = off;
  return p;
}

cudaError_t launch_bin_sort(const sdgs_projected& proj, const sdgs_view& v, const BinPlan& plan,
                            char* ws, const sdgs_bins& out, cudaStream_t st) {
  const int64_t n = plan.n;
  const int tiles_x = tiles_of(v.width), tiles_y = tiles_of(v.height);
  uint32_t* dkeys[2] = {reinterpret_cast<uint32_t*>(ws + plan.off_dkeys[0]),
                        reinterpret_cast<uint32_t*>(ws + plan.off_dkeys[1])};
  uint32_t* dvals[2] = {reinterpret_cast<uint32_t*>(ws + plan.off_dvals[0]),
                        reinterpret_cast<uint32_t*>(ws + plan.off_dvals[1])};
  uint64_t* offsets = reinterpret_cast<uint64_t*>(ws + plan.off_counts);
  uint32_t* hist = reinterpret_cast<uint32_t*>(ws + plan.off_hist);
  uint64_t* partials = reinterpret_cast<uint64_t*>(ws + plan.off_partials);
  const ushort4* rect = reinterpret_cast<const ushort4*>(proj.rect);

  cudaError_t e = cudaMemsetAsync(out.ranges, 0, sizeof(uint32_t) * 2 * (size_t)plan.num_tiles, st);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(out.num_instances, 0, sizeof(int64_t), st);
  if (e != cudaSuccess) return e;
  if (n == 0) return cudaGetLastError();

  const int tb = 256;
  const unsigned gb = (unsigned)((n + tb - 1) / tb);
  // 1. Gaussians by float32 depth (stable; culled ones last).
  depth_keys_kernel<<<gb, tb, 0, st>>>(proj.depth, rect, n, dkeys[0], dvals[0]);
  const int dcur = radix_sort(dkeys, dvals, nullptr, n, n, 32, hist, partials, st);
  const uint32_t* order = dvals[dcur];
  // 2. Instance offsets in depth order; K -> out.num_instances.
  uint32_t* counts = dkeys[dcur ^ 1];
  tile_counts_kernel<<<gb, tb, 0, st>>>(order, rect, n, tiles_x, tiles_y, counts);
  e = exclusive_scan<uint32_t, uint64_t>(counts, n, offsets, partials, out.num_instances, st);
  if (e != cudaSuccess) return e;
  // 3. Duplicate into the buffer that makes the tile passes finish in `out`.
  const int passes = (plan.tile_bits + 7) / 8;
  uint32_t* ikeys[2];
  uint32_t* ivals[2];
  uint32_t* wk = reinterpret_cast<uint32_t*>(ws + plan.off_ikeys);
  uint32_t* wv = reinterpret_cast<uint32_t*>(ws + plan.off_ivals);
  if (passes % 2 == 0) {
    ikeys[0] = out.tile_keys; ivals[0] = out.point_list; ikeys[1] = wk; ivals[1] = wv;
  } else {
    ikeys[0] = wk; ivals[0] = wv; ikeys[1] = out.tile_keys; ivals[1] = out.point_list;
  }
  duplicate_kernel<<<gb, tb, 0, st>>>(order, offsets, rect, tiles_x, tiles_y, n, plan.capacity,
                                      ikeys[0], ivals[0]);
  // 4. Stable sort of the instances by tile id.
  radix_sort(ikeys, ivals, out.num_instances, 0, plan.capacity, plan.tile_bits, hist, partials, st);
  // 5. Tile ranges.
  if (plan.capacity > 0) {
    const unsigned gr = (unsigned)((plan.capacity + tb - 1) / tb);
    ranges_kernel<<<gr, tb, 0, st>>>(out.tile_keys, out.num_instances, plan.capacity,
                                     reinterpret_cast<uint2*>(out.ranges));
  }
  return cudaGetLastError();
}

}  // namespace sdgs
