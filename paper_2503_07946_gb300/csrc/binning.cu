// Tile binning: the stable sort of the (tile << 32 | float32 depth bits) instance keys as an LSD
// sort in two digits -- depth first, then tile -- arranged so that neither pass touches more
// data than it must.
//
// Depth digit: every instance of one Gaussian carries that Gaussian's depth, and instances are
// emitted in the order of the Gaussians.  So the depth passes of an LSD sort over the K instances
// give the same order as a stable radix sort of the n Gaussians by depth (ties keep ascending id)
// followed by emission in that order.  That sort runs over n keys, not K.
//
// Tile digit: one stable counting pass over the depth-ordered Gaussians that writes every
// instance exactly once, straight into its tile's list (see the kernels below).
//
// The depth radix passes are reduce-then-scan with no inter-block waiting: an upsweep writes a
// per-block digit histogram (digit-major), a device-wide exclusive scan turns it into block
// offsets, and a downsweep ranks the block's keys stably (warp match + per-warp counters) and
// scatters them through shared memory so that runs of one digit are written contiguously.
#include <algorithm>

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
                     int64_t cap, int shift, uint32_t* __restrict__ hist, int64_t nblocks,
                     bool block_major) {
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
  if (block_major)
    hist[(int64_t)blockIdx.x * kBins + threadIdx.x] = tot;
  else
    hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kRadixThreads)
radix_downsweep_kernel(const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
                       uint32_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out,
                       const int64_t* nptr, int64_t n_static, int64_t cap, int shift,
                       const uint32_t* __restrict__ hist, int64_t nblocks, bool block_major) {
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
    if (block_major) {
      // raw per-block counts: offset = keys of smaller digits anywhere + this digit in earlier blocks
      uint32_t before = 0, all = 0;
      for (int64_t b = 0; b < nblocks; ++b) {
        const uint32_t c = hist[b * kBins + dg];
        all += c;
        before += (b < (int64_t)blockIdx.x) ? c : 0u;
      }
      uint32_t dtot;
      const uint32_t dincl = block_inclusive_scan<uint32_t, kRadixThreads>(all, &dtot);
      s_gbase[dg] = dincl - all + before;
    } else {
      s_gbase[dg] = hist[(int64_t)dg * nblocks + blockIdx.x];
    }
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
// Up to this many blocks, each downsweep block derives its offsets from the raw per-block
// histograms itself (two kernels per pass); beyond it a device-wide scan runs between them.
constexpr int64_t kFusedScanMaxBlocks = 128;

int radix_sort(uint32_t* keys[2], uint32_t* vals[2], const int64_t* nptr, int64_t n_static,
               int64_t cap, int bits, uint32_t* hist, uint64_t* partials, cudaStream_t st) {
  const int64_t nblocks = (cap + kRadixTile - 1) / kRadixTile;
  int cur = 0;
  if (nblocks == 0) return cur;
  const bool fused = nblocks <= kFusedScanMaxBlocks;
  for (int shift = 0; shift < bits; shift += 8) {
    radix_upsweep_kernel<<<(unsigned)nblocks, kRadixThreads, 0, st>>>(keys[cur], nptr, n_static,
                                                                        cap, shift, hist, nblocks, fused);
    if (!fused)
      exclusive_scan<uint32_t, uint32_t>(hist, (int64_t)kBins * nblocks, hist, partials, nullptr, st);
    radix_downsweep_kernel<<<(unsigned)nblocks, kRadixThreads, 0, st>>>(
        keys[cur], vals[cur], keys[cur ^ 1], vals[cur ^ 1], nptr, n_static, cap, shift, hist,
        nblocks, fused);
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

// ------------------------------------------------------------------------------------------
// Stable counting sort of the instances by tile, in one pass over the depth-sorted Gaussians.
//
// The depth-ordered Gaussians are cut into C contiguous chunks of about equal scatter cost
// (instances / 32 + 1 per Gaussian, running sum split into C equal shares).  (1) Each chunk counts, per tile, how many of its Gaussians' rectangles cover that
// tile, with a 2D difference array in shared memory (four atomics per Gaussian, then prefix sums
// along x and y).  (2) One exclusive scan over the tile-major (tile, chunk) count matrix gives
// every chunk its first output position per tile.  (3) Each chunk walks its Gaussians in depth
// order with one warp: the lanes cover the current Gaussian's rectangle, each writing the
// Gaussian's id at its tile's cursor and advancing it.  Instances of one tile therefore land in
// (depth, id) order, exactly the stable sort by (tile, depth) key.  Per-tile ranges come
// straight from the scanned matrix.
// ------------------------------------------------------------------------------------------

// Rectangles are clipped to the tile grid, so records that come from the caller rather than
// from slice_project can never address a tile outside the image.
__device__ __forceinline__ ushort4 clip_rect(ushort4 r, int tiles_x, int tiles_y) {
  r.x = (unsigned short)min((int)r.x, tiles_x);
  r.z = (unsigned short)min((int)r.z, tiles_x);
  r.y = (unsigned short)min((int)r.y, tiles_y);
  r.w = (unsigned short)min((int)r.w, tiles_y);
  return r;
}

// Scatter cost of each depth-ordered Gaussian in warp steps: one per 32 instances plus one for
// the Gaussian itself.  Chunks are cut at equal shares of the running sum of this cost.
__global__ void work_units_kernel(const uint32_t* __restrict__ order, const ushort4* __restrict__ rect,
                                  int64_t n, int tiles_x, int tiles_y, uint32_t* __restrict__ units) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const ushort4 r = clip_rect(rect[order[s]], tiles_x, tiles_y);
  const int w = (int)r.z - (int)r.x, h = (int)r.w - (int)r.y;
  units[s] = (w > 0 && h > 0) ? (uint32_t)((w * h + 31) / 32 + 1) : 0u;
}

// First s in [0, n) with off[s] >= target (n if none), by a 32-way search over the warp.
__device__ int64_t warp_lower_bound(const uint64_t* __restrict__ off, int64_t n, uint64_t target) {
  const int lane = threadIdx.x & 31;
  int64_t lo = 0, hi = n;  // the answer lies in [lo, hi]; hi == n or off[hi] >= target
  while (hi - lo > 31) {
    const int64_t step = (hi - lo + 31) / 32;
    int64_t p = lo + (int64_t)(lane + 1) * step - 1;
    if (p > hi - 1) p = hi - 1;
    const unsigned b = __ballot_sync(0xffffffffu, off[p] >= target);
    if (b == 0) {
      lo = hi;
      break;
    }
    const int f = __ffs(b) - 1;
    const int64_t pf = min(lo + (int64_t)(f + 1) * step - 1, hi - 1);
    lo = lo + (int64_t)f * step;
    hi = pf;
  }
  const int64_t p = lo + lane;
  const unsigned b = __ballot_sync(0xffffffffu, p >= hi || off[p] >= target);
  return lo + (__ffs(b) - 1);
}

// Gaussian range [s0, s1) of chunk `c` out of `chunks`: the Gaussians whose running cost `off`
// starts inside the chunk's share of `total`.  Executed by a full warp.
__device__ __forceinline__ void chunk_range(const uint64_t* __restrict__ off, int64_t n,
                                            const int64_t* __restrict__ total, int64_t chunks,
                                            int64_t c, int64_t* s0, int64_t* s1) {
  const uint64_t k = (uint64_t)*total;
  uint64_t per = (k + (uint64_t)chunks - 1) / (uint64_t)chunks;
  if (per == 0) per = 1;
  // Targets are clamped to the total: the first Gaussian whose running cost reaches the total
  // starts the culled (zero-cost) tail, which belongs to no chunk.
  const uint64_t t0 = (uint64_t)c * per, t1 = (uint64_t)(c + 1) * per;
  *s0 = warp_lower_bound(off, n, t0 < k ? t0 : k);
  *s1 = warp_lower_bound(off, n, t1 < k ? t1 : k);
}

constexpr int kHistThreads = 256;

__global__ void __launch_bounds__(kHistThreads)
chunk_hist_kernel(const uint32_t* __restrict__ order, const ushort4* __restrict__ rect, int64_t n,
                  const uint64_t* __restrict__ offsets, const int64_t* __restrict__ total, int tiles_x,
                  int tiles_y, int64_t chunks, uint32_t* __restrict__ counts) {
  extern __shared__ int s_diff[];  // (tiles_y + 1) x (tiles_x + 1)
  __shared__ int64_t s_range[2];
  const int W1 = tiles_x + 1, H1 = tiles_y + 1;
  for (int i = threadIdx.x; i < W1 * H1; i += kHistThreads) s_diff[i] = 0;
  if (threadIdx.x < 32) {
    int64_t a, b;
    chunk_range(offsets, n, total, chunks, blockIdx.x, &a, &b);
    if (threadIdx.x == 0) { s_range[0] = a; s_range[1] = b; }
  }
  __syncthreads();
  const int64_t s0 = s_range[0], s1 = s_range[1];
  for (int64_t s = s0 + threadIdx.x; s < s1; s += kHistThreads) {
    const ushort4 r = clip_rect(rect[order[s]], tiles_x, tiles_y);
    if (r.z > r.x && r.w > r.y) {
      atomicAdd(&s_diff[r.y * W1 + r.x], 1);
      atomicAdd(&s_diff[r.y * W1 + r.z], -1);
      atomicAdd(&s_diff[r.w * W1 + r.x], -1);
      atomicAdd(&s_diff[r.w * W1 + r.z], 1);
    }
  }
  __syncthreads();
  // prefix sums along x (one warp per row), then along y (one warp per column)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int row = warp; row < tiles_y; row += kHistThreads / 32) {
    int carry = 0;
    for (int x0 = 0; x0 < tiles_x; x0 += 32) {
      const int x = x0 + lane;
      int v = x < tiles_x ? s_diff[row * W1 + x] : 0;
      v = warp_inclusive_scan(v) + carry;
      if (x < tiles_x) s_diff[row * W1 + x] = v;
      carry = __shfl_sync(0xffffffffu, v, 31);
    }
  }
  __syncthreads();
  for (int x0 = warp * 32; x0 < tiles_x; x0 += kHistThreads) {
    const int x = x0 + lane;
    if (x < tiles_x) {
      int run = 0;
      for (int y = 0; y < tiles_y; ++y) {
        run += s_diff[y * W1 + x];
        counts[(int64_t)(y * tiles_x + x) * chunks + blockIdx.x] = (uint32_t)run;
      }
    }
  }
}

__global__ void __launch_bounds__(32)
chunk_scatter_kernel(const uint32_t* __restrict__ order, const ushort4* __restrict__ rect, int64_t n,
                     const uint64_t* __restrict__ offsets, const int64_t* __restrict__ total, int tiles_x,
                     int tiles_y, int64_t chunks, const uint64_t* __restrict__ base, int64_t cap,
                     uint32_t* __restrict__ point_list, uint32_t* __restrict__ tile_keys) {
  extern __shared__ uint32_t s_cur[];  // one cursor per tile
  const int tiles = tiles_x * tiles_y;
  const int lane = threadIdx.x;
  const int64_t chunk = blockIdx.x;
  int64_t s0, s1;
  chunk_range(offsets, n, total, chunks, chunk, &s0, &s1);
#pragma unroll 8
  for (int t = lane; t < tiles; t += 32) {
    const uint64_t b = base[(int64_t)t * chunks + chunk];
    s_cur[t] = (uint32_t)(b < (uint64_t)cap ? b : (uint64_t)cap);
  }
  __syncwarp();
  for (int64_t sg = s0; sg < s1; sg += 32) {
    // each lane fetches one Gaussian of the group; they are then handled one at a time
    uint32_t g = 0;
    ushort4 r = make_ushort4(0, 0, 0, 0);
    if (sg + lane < s1) {
      g = order[sg + lane];
      r = clip_rect(rect[g], tiles_x, tiles_y);
    }
    unsigned todo = __ballot_sync(0xffffffffu, r.z > r.x && r.w > r.y);
    while (todo) {
      const int i = __ffs(todo) - 1;
      todo &= todo - 1;
      const uint32_t gi = __shfl_sync(0xffffffffu, g, i);
      const int rx0 = __shfl_sync(0xffffffffu, (int)r.x, i);
      const int ry0 = __shfl_sync(0xffffffffu, (int)r.y, i);
      const int w = __shfl_sync(0xffffffffu, (int)r.z, i) - rx0;
      const int h = __shfl_sync(0xffffffffu, (int)r.w, i) - ry0;
      if (w > 0 && h > 0) {
        const int cnt = w * h;
        int dy = lane / w, dx = lane - dy * w;  // position of this lane's first tile
        const int step_y = 32 / w, step_x = 32 - step_y * w;
        for (int k = lane; k < cnt; k += 32) {
          const int t = (ry0 + dy) * tiles_x + rx0 + dx;
          const uint32_t p = s_cur[t];
          s_cur[t] = p + 1;
          if (p < (uint32_t)cap) {
            point_list[p] = gi;
            if (tile_keys != nullptr) tile_keys[p] = (uint32_t)t;
          }
          dx += step_x;
          dy += step_y;
          if (dx >= w) { dx -= w; ++dy; }
        }
      }
      __syncwarp();
    }
  }
}

__global__ void ranges_from_base_kernel(const uint64_t* __restrict__ base, int tiles, int64_t chunks,
                                        const int64_t* __restrict__ total, int64_t cap,
                                        uint2* __restrict__ ranges) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= tiles) return;
  const uint64_t k = (uint64_t)*total;
  const uint64_t st = base[(int64_t)t * chunks];
  const uint64_t en = (t + 1 < tiles) ? base[(int64_t)(t + 1) * chunks] : k;
  ranges[t] = make_uint2((uint32_t)(st < (uint64_t)cap ? st : cap), (uint32_t)(en < (uint64_t)cap ? en : cap));
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Number of counting-sort chunks: enough for parallelism, with the (tile, chunk) matrix kept
// within 4M entries.
int64_t chunk_count(int tiles) {
  int64_t c = (int64_t(4) << 20) / (tiles > 0 ? tiles : 1);
  return c < 128 ? 128 : (c > 1024 ? 1024 : c);
}

}  // namespace

size_t bin_smem_bytes(int width, int height) {
  const size_t hist = sizeof(int) * (size_t)(tiles_of(width) + 1) * (tiles_of(height) + 1);
  const size_t cur = sizeof(uint32_t) * (size_t)tiles_of(width) * tiles_of(height);
  return hist > cur ? hist : cur;
}

BinPlan plan_bins(int64_t n, int64_t capacity, int width, int height) {
  BinPlan p;
  p.n = n;
  p.capacity = capacity;
  p.num_tiles = tiles_of(width) * tiles_of(height);
  p.tile_bits = 0;
  p.chunks = chunk_count(p.num_tiles);
  p.chunk = 0;
  const int64_t nb_d = (n + kRadixTile - 1) / kRadixTile;
  p.hist_blocks = nb_d;
  const int64_t hist_entries = (int64_t)kBins * nb_d;
  const int64_t mat = (int64_t)p.num_tiles * p.chunks;
  const int64_t part_a = (hist_entries + kScanChunk - 1) / kScanChunk;
  const int64_t part_b = (mat + kScanChunk - 1) / kScanChunk;
  const int64_t part_c = (n + kScanChunk - 1) / kScanChunk;
  p.partial_cap = std::max(part_a, std::max(part_b, part_c)) + 1;
  size_t off = 0;
  for (int k = 0; k < 2; ++k) { p.off_dkeys[k] = off; off += align256(sizeof(uint32_t) * n); }
  for (int k = 0; k < 2; ++k) { p.off_dvals[k] = off; off += align256(sizeof(uint32_t) * n); }
  p.off_offsets = off; off += align256(sizeof(uint64_t) * n);
  p.off_counts = off; off += align256(sizeof(uint32_t) * mat);
  p.off_base = off; off += align256(sizeof(uint64_t) * mat);
  p.off_hist = off; off += align256(sizeof(uint32_t) * hist_entries);
  p.off_partials = off; off += align256(sizeof(uint64_t) * p.partial_cap);
  p.off_scalars = off; off += align256(sizeof(int64_t) * 4);
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
  uint64_t* offsets = reinterpret_cast<uint64_t*>(ws + plan.off_offsets);
  uint32_t* counts = reinterpret_cast<uint32_t*>(ws + plan.off_counts);
  uint64_t* base = reinterpret_cast<uint64_t*>(ws + plan.off_base);
  uint32_t* hist = reinterpret_cast<uint32_t*>(ws + plan.off_hist);
  uint64_t* partials = reinterpret_cast<uint64_t*>(ws + plan.off_partials);
  int64_t* total_work = reinterpret_cast<int64_t*>(ws + plan.off_scalars);
  const ushort4* rect = reinterpret_cast<const ushort4*>(proj.rect);

  cudaError_t e;
  if (n == 0) {
    e = cudaMemsetAsync(out.ranges, 0, sizeof(uint32_t) * 2 * (size_t)plan.num_tiles, st);
    if (e != cudaSuccess) return e;
    return cudaMemsetAsync(out.num_instances, 0, sizeof(int64_t), st);
  }
  const int tb = 256;
  const unsigned gb = (unsigned)((n + tb - 1) / tb);
  // 1. Gaussians by float32 depth (stable; culled ones last).
  depth_keys_kernel<<<gb, tb, 0, st>>>(proj.depth, rect, n, dkeys[0], dvals[0]);
  const int dcur = radix_sort(dkeys, dvals, nullptr, n, n, 32, hist, partials, st);
  const uint32_t* order = dvals[dcur];
  // 2. Running scatter cost in depth order, to cut balanced chunks.
  uint32_t* tcount = dkeys[dcur ^ 1];
  work_units_kernel<<<gb, tb, 0, st>>>(order, rect, n, tiles_x, tiles_y, tcount);
  e = exclusive_scan<uint32_t, uint64_t>(tcount, n, offsets, partials, total_work, st);
  if (e != cudaSuccess) return e;
  // 3. Per-chunk tile counts, scanned tile-major: first position of every (tile, chunk).
  const size_t smem = bin_smem_bytes(v.width, v.height);
  e = cudaFuncSetAttribute(chunk_hist_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(chunk_scatter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  chunk_hist_kernel<<<(unsigned)plan.chunks, kHistThreads, smem, st>>>(
      order, rect, n, offsets, total_work, tiles_x, tiles_y, plan.chunks, counts);
  const int64_t mat = (int64_t)plan.num_tiles * plan.chunks;
  e = exclusive_scan<uint32_t, uint64_t>(counts, mat, base, partials, out.num_instances, st);
  if (e != cudaSuccess) return e;
  // 4. Scatter the ids into their tiles' lists; 5. ranges.
  chunk_scatter_kernel<<<(unsigned)plan.chunks, 32, smem, st>>>(
      order, rect, n, offsets, total_work, tiles_x, tiles_y, plan.chunks, base, plan.capacity,
      out.point_list, out.tile_keys);
  ranges_from_base_kernel<<<(plan.num_tiles + tb - 1) / tb, tb, 0, st>>>(
      base, plan.num_tiles, plan.chunks, out.num_instances, plan.capacity, reinterpret_cast<uint2*>(out.ranges));
  return cudaGetLastError();
}

}  // namespace sdgs
