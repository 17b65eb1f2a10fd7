// Tile binning: the stable sort of the (tile << 32 | float32 depth bits) instance keys as an LSD
// sort in two digits, depth first, arranged so that neither digit's passes touch more data than
// they must.
//
// Depth digit: every instance of one Gaussian carries that Gaussian's depth, and instances are
// emitted in the order of the Gaussians.  So the depth passes of an LSD sort over the K instances
// give the same order as a stable radix sort of the n Gaussians by depth (ties keep ascending id)
// followed by emission in that order.  That sort runs over n keys, not K.
//
// Tile digit: the instances, emitted in depth order, are radix-sorted stably by tile id
// (ceil(log2 tiles) bits, in passes of equal width <= 8 bits).  Instances exist only inside the
// per-row spans of tiles a Gaussian may reach (tile_reach.cuh).
//
// Each radix pass is one kernel (digit histograms of all passes are accumulated while the keys are
// produced): a block ranks its tile of keys stably, finds the keys of each digit in earlier tiles
// by a decoupled look-back (bounded waits), and writes each digit's run contiguously.
#include <algorithm>

#include "common.cuh"
#include "tile_reach.cuh"

namespace sdgs {

namespace {

constexpr int kRadixThreads = 256;
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
  griddep_wait();
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
  griddep_wait();
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
  griddep_wait();
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
  cudaError_t e = cudaSuccess;
  if (nb > 0) e = launch_pdl(scan_reduce_kernel<TIn, TOut>, dim3((unsigned)nb), dim3(kScanThreads), 0, st, in, n, part);
  if (e == cudaSuccess) e = launch_pdl(scan_partials_kernel<TOut>, dim3(1), dim3(1024), 0, st, part, nb, total_out);
  if (e == cudaSuccess && nb > 0)
    e = launch_pdl(scan_down_kernel<TIn, TOut>, dim3((unsigned)nb), dim3(kScanThreads), 0, st, in, n, part, out);
  return e;
}

// ------------------------------------------------------------------------------------------
// Radix pass kernels (8-bit digit at `shift`).
// ------------------------------------------------------------------------------------------

// Lanes of the warp whose digit equals this lane's (d has `width` bits; lanes with !valid are in
// no lane's set): one ballot per digit bit.
template <bool FULL>
__device__ __forceinline__ unsigned digit_peers(uint32_t d, bool valid, int width) {
  unsigned peers = FULL ? 0xffffffffu : __ballot_sync(0xffffffffu, valid);
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    if (b < width) {  // uniform over the warp
      const bool bit = (d >> b) & 1u;
      const unsigned m = __ballot_sync(0xffffffffu, bit);
      peers &= bit ? m : ~m;
    }
  }
  return peers;
}

// ------------------------------------------------------------------------------------------
// LSD radix sort of (key, value) pairs: one histogram kernel for every digit, then one kernel per
// digit.  A sort block ranks its tile of keys stably (per-warp digit counters; lanes with equal
// digits found by match or by one ballot per digit bit), finds the keys of each digit in all
// earlier tiles by a decoupled look-back over the per-tile status words, and writes each digit's
// run of keys contiguously through shared memory.  Tiles are numbered by an atomic ticket taken
// when a block starts, so a block only ever waits on blocks that are already running; every wait
// is bounded (kLookbackSpins), after which the block flags an error and carries on.
// ------------------------------------------------------------------------------------------

constexpr uint32_t kStatusAggregate = 1u << 30;  // this tile's own count of the digit
constexpr uint32_t kStatusInclusive = 2u << 30;  // count of the digit in tiles 0 .. this one
constexpr uint32_t kStatusCount = (1u << 30) - 1u;
constexpr int kLookbackSpins = 1 << 20;
constexpr int kLookbackWindow = 8;
constexpr int kMaxPasses = 4;

__global__ void __launch_bounds__(kRadixThreads)
digit_hist_kernel(const uint32_t* __restrict__ keys, const int64_t* nptr, int64_t n_static, int64_t cap,
                  int passes, int width, uint32_t* __restrict__ hist) {
  griddep_wait();
  __shared__ uint32_t s_hist[kMaxPasses][kBins];
  for (int i = threadIdx.x; i < kMaxPasses * kBins; i += kRadixThreads) (&s_hist[0][0])[i] = 0;
  __syncthreads();
  const int64_t n = element_count(nptr, n_static, cap);
  const uint32_t dmask = (1u << width) - 1u;
  for (int64_t i = (int64_t)blockIdx.x * kRadixThreads + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * kRadixThreads) {
    const uint32_t k = keys[i];
    for (int p = 0; p < passes; ++p) atomicAdd(&s_hist[p][(k >> (p * width)) & dmask], 1u);
  }
  __syncthreads();
  for (int p = 0; p < passes; ++p) {
    const uint32_t c = s_hist[p][threadIdx.x];
    if (c) atomicAdd(&hist[p * kBins + threadIdx.x], c);
  }
}

__device__ __forceinline__ uint32_t load_status(const uint32_t* p) {
  return *reinterpret_cast<const volatile uint32_t*>(p);
}
__device__ __forceinline__ void store_status(uint32_t* p, uint32_t v) {
  *reinterpret_cast<volatile uint32_t*>(p) = v;
}

// Loads a warp's ITEMS rows of 32 keys and ranks each key among the warp's keys with the same
// digit (stable: earlier rows, then lower lanes, first), counting them in s_whist[warp].  FULL: the
// whole tile is in range, so no key needs a bound check.
template <int ITEMS, bool FULL>
__device__ __forceinline__ void load_and_rank(const uint32_t* __restrict__ keys_in, int64_t wbase, int64_t n,
                                              int shift, int width, uint32_t* whist, uint32_t key[ITEMS],
                                              uint32_t rank[ITEMS]) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = lanemask_lt();
  const uint32_t dmask = (1u << width) - 1u;
#pragma unroll
  for (int r = 0; r < ITEMS; ++r) {
    const int64_t idx = wbase + r * 32 + lane;
    key[r] = (FULL || idx < n) ? keys_in[idx] : 0u;
  }
#pragma unroll
  for (int r = 0; r < ITEMS; ++r) {
    const bool valid = FULL || wbase + r * 32 + lane < n;
    const uint32_t d = (key[r] >> shift) & dmask;
    const unsigned peers = width >= 8 ? (__match_any_sync(0xffffffffu, valid ? d : 0x100u) &
                                         (FULL ? 0xffffffffu : __ballot_sync(0xffffffffu, valid)))
                                      : digit_peers<FULL>(d, valid, width);
    const uint32_t before = valid ? whist[d] : 0u;
    __syncwarp();
    if (valid && lane == __ffs(peers) - 1) whist[d] = before + __popc(peers);
    __syncwarp();
    rank[r] = before + __popc(peers & lt);
  }
}

template <int ITEMS>
__global__ void __launch_bounds__(kRadixThreads, ITEMS >= 12 ? 4 : 6)
onesweep_kernel(const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
                uint32_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out, const int64_t* nptr,
                int64_t n_static, int64_t cap, int shift, int width, const uint32_t* __restrict__ digit_hist,
                uint32_t* status, uint32_t* ticket, uint32_t* err) {
  griddep_wait();
  constexpr int TILE = kRadixThreads * ITEMS;
  __shared__ uint32_t s_keys[TILE];
  __shared__ uint32_t s_vals[TILE];
  __shared__ uint32_t s_whist[kRadixWarps][kBins];
  __shared__ uint32_t s_dstart[kBins];
  __shared__ uint32_t s_gbase[kBins];
  __shared__ uint32_t s_tile;
  if (threadIdx.x == 0) s_tile = atomicAdd(ticket, 1u);
  for (int i = threadIdx.x; i < kRadixWarps * kBins; i += kRadixThreads) (&s_whist[0][0])[i] = 0;
  __syncthreads();
  const int64_t tile = s_tile;
  const int64_t n = element_count(nptr, n_static, cap);
  const int64_t base = tile * TILE;
  if (base >= n) return;  // so do all later tiles: nobody waits on this one

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t dmask = (1u << width) - 1u;
  const int64_t wbase = base + (int64_t)warp * 32 * ITEMS;
  const bool full = base + TILE <= n;  // uniform over the block
  uint32_t key[ITEMS], rank[ITEMS];
  if (full) load_and_rank<ITEMS, true>(keys_in, wbase, n, shift, width, s_whist[warp], key, rank);
  else load_and_rank<ITEMS, false>(keys_in, wbase, n, shift, width, s_whist[warp], key, rank);
  __syncthreads();
  {
    const int dg = threadIdx.x;
    uint32_t run = 0;  // this tile's keys with digit dg
#pragma unroll
    for (int w = 0; w < kRadixWarps; ++w) {
      const uint32_t c = s_whist[w][dg];
      s_whist[w][dg] = run;
      run += c;
    }
    uint32_t* mine = status + tile * kBins + dg;
    const bool used = dg <= (int)dmask;  // digits of `width` bits: the other bins stay empty
    if (used) store_status(mine, (tile == 0 ? kStatusInclusive : kStatusAggregate) | run);
    uint32_t before = 0;  // keys with digit dg in tiles 0 .. tile - 1
    int spins = 0;
    // Wait for the nearest unresolved tile (one load per poll, with a short sleep), then take up
    // to kLookbackWindow - 1 further tiles from one round of parallel loads, nearest first, until
    // an inclusive count or a tile that has published nothing yet.
    for (int64_t j = used ? tile - 1 : -1; j >= 0;) {
      const uint32_t near = load_status(status + j * kBins + dg);
      if ((near & ~kStatusCount) == 0u) {
        if (++spins > kLookbackSpins) {
          atomicOr(err, 1u);
          break;
        }
        __nanosleep(32);
        continue;
      }
      before += near & kStatusCount;
      if (near & kStatusInclusive) break;
      --j;
      uint32_t st[kLookbackWindow - 1];
#pragma unroll
      for (int w = 0; w < kLookbackWindow - 1; ++w) st[w] = j - w >= 0 ? load_status(status + (j - w) * kBins + dg) : 0u;
      bool done = false, stop = false;
#pragma unroll
      for (int w = 0; w < kLookbackWindow - 1; ++w) {
        if (done || stop || j < 0) continue;
        if ((st[w] & ~kStatusCount) == 0u) {
          stop = true;  // not published yet: poll it next
          continue;
        }
        before += st[w] & kStatusCount;
        if (st[w] & kStatusInclusive) done = true;
        else --j;
      }
      if (done) break;
    }
    if (used && tile > 0) store_status(mine, kStatusInclusive | (before + run));
    uint32_t tot;
    const uint32_t incl = block_inclusive_scan<uint32_t, kRadixThreads>(run, &tot);
    s_dstart[dg] = incl - run;
    const uint32_t all = digit_hist[dg];
    const uint32_t gincl = block_inclusive_scan<uint32_t, kRadixThreads>(all, &tot);
    s_gbase[dg] = gincl - all + before;
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < ITEMS; ++r) {
    const int64_t idx = wbase + r * 32 + lane;
    if (full || idx < n) {
      const uint32_t d = (key[r] >> shift) & dmask;
      const uint32_t pos = s_dstart[d] + s_whist[warp][d] + rank[r];
      s_keys[pos] = key[r];
      s_vals[pos] = vals_in[idx];
    }
  }
  __syncthreads();
  if (full) {
#pragma unroll
    for (int r = 0; r < ITEMS; ++r) {
      const int i = r * kRadixThreads + threadIdx.x;
      const uint32_t k = s_keys[i];
      const uint32_t d = (k >> shift) & dmask;
      const uint32_t g = s_gbase[d] + (uint32_t)i - s_dstart[d];
      keys_out[g] = k;
      vals_out[g] = s_vals[i];
    }
  } else {
    const int cnt = (int)(n - base);
    for (int i = threadIdx.x; i < cnt; i += kRadixThreads) {
      const uint32_t k = s_keys[i];
      const uint32_t d = (k >> shift) & dmask;
      const uint32_t g = s_gbase[d] + (uint32_t)i - s_dstart[d];
      keys_out[g] = k;
      vals_out[g] = s_vals[i];
    }
  }
}

int radix_digit_width(int bits) {
  const int passes = (bits + 7) / 8;
  return passes > 0 ? (bits + passes - 1) / passes : 8;
}

int radix_pass_count(int bits) {
  int k = 0;
  for (int shift = 0; shift < bits; shift += radix_digit_width(bits)) ++k;
  return k;
}

// Keys per sort block for `cap` slots: the largest tile (12, 8 or 4 keys per thread) that still
// gives two blocks per SM, so that small sorts are not latency-bound on a few blocks.
int sort_items(int64_t cap) {
  const int64_t want = 2 * 152;
  if ((cap + 12 * kRadixThreads - 1) / (12 * kRadixThreads) >= want) return 12;
  if ((cap + 8 * kRadixThreads - 1) / (8 * kRadixThreads) >= want) return 8;
  return 4;
}

int64_t sort_blocks(int64_t cap) {
  const int64_t tile = (int64_t)sort_items(cap) * kRadixThreads;
  return (cap + tile - 1) / tile;
}

// Scratch of one sort: per-digit histograms, tickets, status words.
size_t sort_scratch_bytes(int64_t cap, int bits) {
  return sizeof(uint32_t) * ((size_t)kMaxPasses * kBins + kMaxPasses +
                             (size_t)radix_pass_count(bits) * sort_blocks(cap) * kBins);
}

// Sorts (keys, vals) by bits [0, bits) in ceil(bits / 8) passes of equal digit width (at most 8
// bits: fewer, longer digit runs per block make the writes more contiguous), ping-ponging between
// buffers 0 and 1; returns the index of the buffer that holds the result.  The element count is
// *nptr (clipped to cap) when nptr is not NULL, else n_static; launches are sized by cap.
// `scratch` holds sort_scratch_bytes(cap, bits); `err` is set if a look-back gave up.
// Zeroes a sort's scratch (histograms, tickets, status words).
cudaError_t sort_clear(uint32_t* scratch, int64_t cap, int bits, cudaStream_t st) {
  return cudaMemsetAsync(scratch, 0, sort_scratch_bytes(cap, bits), st);
}

// Adds the digits of every pass of the warp's valid keys to a block's shared histograms
// (s_hist[pass][digit]) with one add per run of adjacent valid lanes with equal digits (runs are
// common: the top digit of nearby depths, the high digit of a row of tiles).  All 32 lanes call.
__device__ __forceinline__ void count_digits(uint32_t (*s_hist)[kBins], uint32_t key, bool valid, int passes,
                                             int width) {
  const uint32_t dmask = (1u << width) - 1u;
  const unsigned live = __ballot_sync(0xffffffffu, valid);
  if (live == 0u) return;
  const int lane = threadIdx.x & 31;
  const bool prev_live = lane > 0 && ((live >> (lane - 1)) & 1u);
  for (int p = 0; p < passes; ++p) {
    const uint32_t d = (key >> (p * width)) & dmask;
    const uint32_t prev = __shfl_up_sync(0xffffffffu, d, 1);
    const bool head = valid && !(prev_live && prev == d);
    const unsigned ends = __ballot_sync(0xffffffffu, head) | ~live;  // a run stops at these lanes
    if (head) {
      const unsigned after = lane < 31 ? (ends >> (lane + 1)) : 0u;
      const uint32_t len = after ? (uint32_t)__ffs(after) : (uint32_t)(32 - lane);
      atomicAdd(&s_hist[p][d], len);
    }
  }
}

__device__ __forceinline__ void flush_digits(const uint32_t (*s_hist)[kBins], int passes, uint32_t* hist) {
  for (int i = threadIdx.x; i < passes * kBins; i += blockDim.x) {
    const uint32_t c = s_hist[i / kBins][i % kBins];
    if (c) atomicAdd(&hist[i], c);
  }
}

// With hist_ready, the caller has cleared the scratch (sort_clear) and accumulated the digit
// histograms of all keys into its first kMaxPasses * kBins words while producing them.
int radix_sort(uint32_t* keys[2], uint32_t* vals[2], const int64_t* nptr, int64_t n_static,
               int64_t cap, int bits, uint32_t* scratch, uint32_t* err, bool hist_ready, cudaStream_t st) {
  int cur = 0;
  if (cap <= 0 || bits <= 0) return cur;
  const int width = radix_digit_width(bits);
  const int passes = radix_pass_count(bits);
  const int items = sort_items(cap);
  const int64_t nblocks = sort_blocks(cap);
  uint32_t* hist = scratch;
  uint32_t* tickets = hist + kMaxPasses * kBins;
  uint32_t* status = tickets + kMaxPasses;
  if (!hist_ready) {
    sort_clear(scratch, cap, bits, st);
    const int64_t hist_blocks = std::min<int64_t>((cap + kRadixThreads - 1) / kRadixThreads, 4 * 152);
    digit_hist_kernel<<<(unsigned)hist_blocks, kRadixThreads, 0, st>>>(keys[0], nptr, n_static, cap, passes,
                                                                       width, hist);
  }
  for (int p = 0; p < passes; ++p) {
    uint32_t* stp = status + (size_t)p * nblocks * kBins;
    const int shift = p * width;
    auto* kern = items == 12 ? onesweep_kernel<12> : items == 8 ? onesweep_kernel<8> : onesweep_kernel<4>;
    launch_pdl(kern, dim3((unsigned)nblocks), dim3(kRadixThreads), 0, st, keys[cur], vals[cur], keys[cur ^ 1],
               vals[cur ^ 1], nptr, n_static, cap, shift, width, hist + p * kBins, stp, tickets + p, err);
    cur ^= 1;
  }
  return cur;
}

// ------------------------------------------------------------------------------------------
// Binning-specific kernels.
// ------------------------------------------------------------------------------------------

// Zeroes the words binning accumulates into or reads before writing: the error word, the tile
// ranges and the instance count (when there are no Gaussians) and both sorts' scratch.  One kernel
// instead of several memsets keeps the render's launches a chain of kernels.
struct ClearJob {
  uint32_t* ptr[5];
  size_t words[5];
};

__global__ void __launch_bounds__(256) clear_kernel(const ClearJob job) {
  griddep_wait();
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (int k = 0; k < 5; ++k) {
    uint32_t* p = job.ptr[k];
    if (p == nullptr) continue;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < job.words[k]; i += stride) p[i] = 0u;
  }
}

// Depth keys of the Gaussians (culled ones last) and their digit histograms for the depth sort.
__global__ void __launch_bounds__(kRadixThreads)
depth_keys_kernel(const float* __restrict__ depth, const ushort4* __restrict__ rect, int64_t n,
                  uint32_t* __restrict__ keys, uint32_t* __restrict__ vals, uint32_t* __restrict__ hist) {
  griddep_wait();
  __shared__ uint32_t s_hist[kMaxPasses][kBins];
  for (int i = threadIdx.x; i < kMaxPasses * kBins; i += kRadixThreads) (&s_hist[0][0])[i] = 0;
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * kRadixThreads + threadIdx.x;
  uint32_t k = 0;
  if (i < n) {
    const ushort4 r = rect[i];
    const bool vis = r.z > r.x && r.w > r.y;
    k = vis ? __float_as_uint(depth[i]) : 0xffffffffu;  // visible depths are positive
    keys[i] = k;
    vals[i] = (uint32_t)i;
  }
  count_digits(s_hist, k, i < n, 4, 8);
  __syncthreads();
  flush_digits(s_hist, 4, hist);
}

// ------------------------------------------------------------------------------------------
// Instances in depth order, then a stable sort on the tile digit.
//
// Each depth-ordered Gaussian walks the rows of its rectangle and takes one span of tiles per row
// from the reachability rule (tile_reach.cuh): a first pass counts the kept tiles, an exclusive
// scan gives each Gaussian its first instance, and a second pass writes its (tile id, Gaussian
// id) pairs contiguously, row-major.  The radix passes over the tile id then make the order
// (tile, depth, id).
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

// The tested tiles of a block of kWalkThreads consecutive depth-ordered Gaussians form one
// sequence -- Gaussian-major, each tested rectangle row-major -- cut into 32-tile words that the
// block's warps share, so a few large rectangles do not leave one warp with all the work.
constexpr int kSpanThreads = 256;

// Kept tiles of each depth-ordered Gaussian (one thread each): its rectangle (clipped to the grid)
// row by row, each row's span from the reachability rule (tile_reach.cuh).
__global__ void __launch_bounds__(kSpanThreads)
span_count_kernel(const uint32_t* __restrict__ order, const ushort4* __restrict__ rect,
                  const float2* __restrict__ mean2d, const float4* __restrict__ conic_opacity, int64_t n,
                  int tiles_x, int tiles_y, uint32_t* __restrict__ counts) {
  griddep_wait();
  const int64_t s = (int64_t)blockIdx.x * kSpanThreads + threadIdx.x;
  if (s >= n) return;
  const uint32_t g = order[s];
  const ushort4 r = clip_rect(rect[g], tiles_x, tiles_y);
  uint32_t c = 0;
  if (r.z > r.x && r.w > r.y) {
    const SpanRule rule = span_setup(mean2d[g], conic_opacity[g]);
    int y0, y1;
    span_rows(rule, r.y, r.w, &y0, &y1);
    for (int ty = y0; ty < y1; ++ty) {
      int x0, x1;
      span_cols(rule, ty, r.x, r.z, &x0, &x1);
      c += (uint32_t)(x1 - x0);
    }
  }
  counts[s] = c;
}

// Digit histograms of the tile ids of a row span id0 .. id0 + len - 1 for the tile sort.  Pass 0
// (the low digit) cycles through its 2^width values along consecutive ids, so each value gets
// floor(len / 2^width) plus one over a cyclic range: a per-block constant and a cyclic difference
// array (at most four adds instead of len).  Higher passes are constant along runs of 2^(p width)
// ids: one add per run.
struct DigitAcc {
  uint32_t (*hist)[kBins];  // passes >= 1
  int32_t* diff0;           // [kBins + 1] difference array of pass 0
  uint32_t* all0;           // added to every pass-0 digit
};

__device__ __forceinline__ void count_span_digits(const DigitAcc& acc, uint32_t id0, uint32_t len, int passes,
                                                  int width) {
  if (passes == 0 || len == 0) return;
  const uint32_t period = 1u << width, dmask = period - 1u;
  const uint32_t full = len >> width, rem = len & dmask;
  if (full) atomicAdd(acc.all0, full);
  if (rem) {
    const uint32_t d0 = id0 & dmask, d1 = d0 + rem;
    atomicAdd(&acc.diff0[d0], 1);
    if (d1 <= period) {
      atomicAdd(&acc.diff0[d1], -1);
    } else {
      atomicAdd(&acc.diff0[period], -1);
      atomicAdd(&acc.diff0[0], 1);
      atomicAdd(&acc.diff0[d1 - period], -1);
    }
  }
  for (int p = 1; p < passes; ++p) {
    const int sh = p * width;
    uint32_t id = id0;
    const uint32_t end = id0 + len;
    while (id < end) {
      const uint32_t d = (id >> sh) & dmask;
      const uint32_t next = min(end, ((id >> sh) + 1u) << sh);  // first id with the next digit value
      atomicAdd(&acc.hist[p][d], next - id);
      id = next;
    }
  }
}

constexpr uint32_t kBigInstances = 32;  // above this a Gaussian is written by its whole warp

__device__ __forceinline__ SpanRule shfl_rule(const SpanRule& q, int src) {
  SpanRule o;
  o.u = __shfl_sync(0xffffffffu, q.u, src);
  o.v = __shfl_sync(0xffffffffu, q.v, src);
  o.a = __shfl_sync(0xffffffffu, q.a, src);
  o.b = __shfl_sync(0xffffffffu, q.b, src);
  o.det = __shfl_sync(0xffffffffu, q.det, src);
  o.aQ = __shfl_sync(0xffffffffu, q.aQ, src);
  o.hx = 0.f;  // not used past setup
  o.reach_y = __shfl_sync(0xffffffffu, q.reach_y, src);
  o.dyr = __shfl_sync(0xffffffffu, q.dyr, src);
  o.padx = __shfl_sync(0xffffffffu, q.padx, src);
  o.mode = __shfl_sync(0xffffffffu, q.mode, src);
  return o;
}

// Writes each depth-ordered Gaussian's (tile id, Gaussian id) pairs from its first instance,
// row-major over its spans, and accumulates the tile-digit histograms of what it writes.  A
// Gaussian with at most kBigInstances instances is written by its own thread (runs stored four
// at a time when keys and vals are 16-byte aligned, `vec`); larger ones are then written by the
// whole warp one at a time -- lanes take 32 rows, a warp scan places their spans, and the lanes
// store consecutive instances -- so that one large Gaussian does not hold up its warp.
// Positions >= cap are dropped.
__global__ void __launch_bounds__(kSpanThreads)
span_emit_kernel(const uint32_t* __restrict__ order, const ushort4* __restrict__ rect,
                 const float2* __restrict__ mean2d, const float4* __restrict__ conic_opacity, int64_t n,
                 int tiles_x, int tiles_y, const uint64_t* __restrict__ first, const uint32_t* __restrict__ counts,
                 int64_t cap, uint32_t* __restrict__ keys, uint32_t* __restrict__ vals, bool vec, int passes,
                 int width, uint32_t* __restrict__ hist) {
  griddep_wait();
  __shared__ uint32_t s_hist[kMaxPasses][kBins];
  __shared__ int32_t s_diff0[kBins + 1];
  __shared__ uint32_t s_all0;
  for (int i = threadIdx.x; i < kMaxPasses * kBins; i += kSpanThreads) (&s_hist[0][0])[i] = 0;
  for (int i = threadIdx.x; i <= kBins; i += kSpanThreads) s_diff0[i] = 0;
  if (threadIdx.x == 0) s_all0 = 0;
  __syncthreads();
  const DigitAcc acc{s_hist, s_diff0, &s_all0};
  const int64_t s = (int64_t)blockIdx.x * kSpanThreads + threadIdx.x;
  const int lane = threadIdx.x & 31;
  uint32_t g = 0;
  ushort4 r = make_ushort4(0, 0, 0, 0);
  SpanRule rule;
  rule.mode = 2;
  int y0 = 0, y1 = 0;
  uint64_t pos = 0;
  bool live = false, big = false;
  if (s < n) {
    pos = first[s];
    const uint32_t cnt = counts[s];
    if (cnt > 0 && pos < (uint64_t)cap) {
      g = order[s];
      r = clip_rect(rect[g], tiles_x, tiles_y);
      rule = span_setup(mean2d[g], conic_opacity[g]);
      span_rows(rule, r.y, r.w, &y0, &y1);
      live = true;
      big = cnt > kBigInstances;
    }
  }
  if (live && !big) {
    const uint4 g4 = make_uint4(g, g, g, g);
    for (int ty = y0; ty < y1 && pos < (uint64_t)cap; ++ty) {
      int x0, x1;
      span_cols(rule, ty, r.x, r.z, &x0, &x1);
      const int64_t room = cap - (int64_t)pos;
      const uint32_t len = (uint32_t)((int64_t)(x1 - x0) < room ? (int64_t)(x1 - x0) : room);
      const uint32_t id0 = (uint32_t)ty * (uint32_t)tiles_x + (uint32_t)x0;
      uint32_t k = 0;
      if (vec) {
        for (; k < len && ((pos + k) & 3u); ++k) {
          keys[pos + k] = id0 + k;
          vals[pos + k] = g;
        }
        for (; k + 4 <= len; k += 4) {
          const uint32_t id = id0 + k;
          *reinterpret_cast<uint4*>(keys + pos + k) = make_uint4(id, id + 1, id + 2, id + 3);
          *reinterpret_cast<uint4*>(vals + pos + k) = g4;
        }
      }
      for (; k < len; ++k) {
        keys[pos + k] = id0 + k;
        vals[pos + k] = g;
      }
      count_span_digits(acc, id0, len, passes, width);
      pos += len;
    }
  }
  for (unsigned bigs = __ballot_sync(0xffffffffu, big); bigs != 0u; bigs &= bigs - 1u) {  // uniform
    const int i = __ffs(bigs) - 1;
    const SpanRule q = shfl_rule(rule, i);
    const uint32_t qg = __shfl_sync(0xffffffffu, g, i);
    const int qx0 = __shfl_sync(0xffffffffu, (int)r.x, i), qx1 = __shfl_sync(0xffffffffu, (int)r.z, i);
    const int qy0 = __shfl_sync(0xffffffffu, y0, i), qy1 = __shfl_sync(0xffffffffu, y1, i);
    uint64_t qpos = __shfl_sync(0xffffffffu, pos, i);
    for (int rb = qy0; rb < qy1; rb += 32) {
      const int ty = rb + lane;
      int x0 = 0, x1 = 0;
      if (ty < qy1) span_cols(q, ty, qx0, qx1, &x0, &x1);
      const uint32_t len = (uint32_t)(x1 - x0);
      const uint32_t incl = warp_inclusive_scan(len);
      const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
      const int64_t rstart = (int64_t)qpos + (int64_t)(incl - len);
      const int64_t room = cap - rstart;
      const uint32_t written = room <= 0 ? 0u : (room < (int64_t)len ? (uint32_t)room : len);
      count_span_digits(acc, (uint32_t)ty * (uint32_t)tiles_x + (uint32_t)x0, written, passes, width);
      for (uint32_t j0 = 0; j0 < total; j0 += 32) {
        const uint32_t j = j0 + lane;
        int rl = 0;  // the row lane holding instance j: the first lane whose inclusive count exceeds j
#pragma unroll
        for (int step = 16; step >= 1; step >>= 1) {
          const uint32_t v = __shfl_sync(0xffffffffu, incl, rl + step - 1);
          if (v <= j) rl += step;
        }
        const uint32_t r_excl = __shfl_sync(0xffffffffu, incl - len, rl);
        const int r_x0 = __shfl_sync(0xffffffffu, x0, rl);
        const uint64_t p = qpos + j;
        if (j < total && p < (uint64_t)cap) {
          keys[p] = (uint32_t)(rb + rl) * (uint32_t)tiles_x + (uint32_t)(r_x0 + (int)(j - r_excl));
          vals[p] = qg;
        }
      }
      qpos += total;
      if (qpos >= (uint64_t)cap) break;  // uniform
    }
  }
  __syncthreads();
  if (passes > 0) {  // pass 0 from the difference array: a running sum over the digits
    if (threadIdx.x < 32) {
      const int period = 1 << width;
      int carry = 0;
      for (int d0 = 0; d0 < period; d0 += 32) {
        const int d = d0 + lane;
        const int v = d < period ? s_diff0[d] : 0;
        const int incl = warp_inclusive_scan(v) + carry;
        if (d < period) s_hist[0][d] = (uint32_t)incl + s_all0;
        carry = __shfl_sync(0xffffffffu, incl, 31);
      }
    }
    __syncthreads();
  }
  flush_digits(s_hist, passes, hist);
}

// First position in keys[0, n) (sorted) whose key is >= t, found by the calling warp: each round
// probes 32 evenly spaced positions of [lo, hi) and keeps the part between the last probe below t
// and the first probe at or above it (32 times shorter), until [lo, hi) is empty.  All 32 lanes
// call; every lane returns the answer.
__device__ __forceinline__ int64_t warp_lower_bound(const uint32_t* __restrict__ keys, int64_t n, uint32_t t) {
  const int lane = threadIdx.x & 31;
  int64_t lo = 0, hi = n;  // keys before lo are < t; keys from hi on are >= t
  while (hi > lo) {
    const int64_t step = (hi - lo + 31) / 32;
    const int64_t p = lo + (int64_t)lane * step;
    const bool below = p < hi && keys[p] < t;
    const int c = __popc(__ballot_sync(0xffffffffu, below));  // the probes below t are a prefix
    const int64_t nhi = lo + (int64_t)c * step;
    lo = c > 0 ? lo + (int64_t)(c - 1) * step + 1 : lo;
    hi = nhi < hi ? nhi : hi;
  }
  return lo;
}

// ranges[t] = [first, end) of tile t in the sorted keys, (0, 0) for a tile without instances; one
// warp per tile.
__global__ void ranges_kernel(const uint32_t* __restrict__ keys, const int64_t* nptr, int64_t cap,
                              int num_tiles, uint2* __restrict__ ranges) {
  griddep_wait();
  const int64_t n = element_count(nptr, 0, cap);
  const int t = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (t >= num_tiles) return;  // whole warps
  const int64_t a = warp_lower_bound(keys, n, (uint32_t)t);
  const int64_t b = warp_lower_bound(keys, n, (uint32_t)t + 1u);
  if ((threadIdx.x & 31) == 0) ranges[t] = b > a ? make_uint2((uint32_t)a, (uint32_t)b) : make_uint2(0u, 0u);
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

BinPlan plan_bins(int64_t n, int64_t capacity, int width, int height) {
  BinPlan p;
  p.n = n;
  p.capacity = capacity;
  p.num_tiles = tiles_of(width) * tiles_of(height);
  int bits = 0;
  while ((int64_t(1) << bits) < p.num_tiles) ++bits;
  p.tile_bits = bits;
  p.partial_cap = (n + kScanChunk - 1) / kScanChunk + 1;
  size_t off = 0;
  for (int k = 0; k < 2; ++k) { p.off_dkeys[k] = off; off += align256(sizeof(uint32_t) * n); }
  for (int k = 0; k < 2; ++k) { p.off_dvals[k] = off; off += align256(sizeof(uint32_t) * n); }
  p.off_first = off; off += align256(sizeof(uint64_t) * n);
  p.off_ikeys[0] = off; off += align256(sizeof(uint32_t) * capacity);
  p.off_ikeys[1] = off; off += align256(sizeof(uint32_t) * capacity);
  p.off_ivals = off; off += align256(sizeof(uint32_t) * capacity);
  p.off_err = off; off += 256;
  p.off_sort_d = off; off += align256(sort_scratch_bytes(n, 32));
  p.off_sort_t = off; off += align256(sort_scratch_bytes(capacity, bits));
  p.off_partials = off; off += align256(sizeof(uint64_t) * p.partial_cap);
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
  uint64_t* first = reinterpret_cast<uint64_t*>(ws + plan.off_first);
  uint32_t* sort_d = reinterpret_cast<uint32_t*>(ws + plan.off_sort_d);
  uint32_t* sort_t = reinterpret_cast<uint32_t*>(ws + plan.off_sort_t);
  uint32_t* err = reinterpret_cast<uint32_t*>(ws + plan.off_err);
  uint64_t* partials = reinterpret_cast<uint64_t*>(ws + plan.off_partials);
  const ushort4* rect = reinterpret_cast<const ushort4*>(proj.rect);
  const float2* m2 = reinterpret_cast<const float2*>(proj.mean2d);
  const float4* co = reinterpret_cast<const float4*>(proj.conic_opacity);

  ClearJob clear;
  // (with Gaussians, the ranges kernel writes every tile's range)
  clear.ptr[0] = n == 0 ? out.ranges : nullptr; clear.words[0] = 2 * (size_t)plan.num_tiles;
  clear.ptr[1] = err; clear.words[1] = 1;
  clear.ptr[2] = n == 0 ? reinterpret_cast<uint32_t*>(out.num_instances) : nullptr; clear.words[2] = 2;
  clear.ptr[3] = n > 0 ? sort_d : nullptr; clear.words[3] = sort_scratch_bytes(n, 32) / 4;
  clear.ptr[4] = n > 0 ? sort_t : nullptr; clear.words[4] = sort_scratch_bytes(plan.capacity, plan.tile_bits) / 4;
  size_t most = 0;
  for (int k = 0; k < 5; ++k) most = std::max(most, clear.ptr[k] ? clear.words[k] : 0);
  const unsigned gc = (unsigned)std::max<size_t>(1, std::min<size_t>((most + 255) / 256, 4 * 152));
  cudaError_t e = launch_pdl(clear_kernel, dim3(gc), dim3(256), 0, st, clear);
  if (e != cudaSuccess || n == 0) return e;
  const unsigned gb = (unsigned)((n + kRadixThreads - 1) / kRadixThreads);
  // 1. Gaussians by float32 depth (stable; culled ones last).
  e = launch_pdl(depth_keys_kernel, dim3(gb), dim3(kRadixThreads), 0, st, proj.depth, rect, n, dkeys[0], dvals[0],
                 sort_d);
  if (e != cudaSuccess) return e;
  const int dcur = radix_sort(dkeys, dvals, nullptr, n, n, 32, sort_d, err, true, st);
  const uint32_t* order = dvals[dcur];
  // 2. Kept tiles per Gaussian (row spans); first instance of each; K.
  uint32_t* counts = dkeys[dcur ^ 1];
  const unsigned gs = (unsigned)((n + kSpanThreads - 1) / kSpanThreads);
  e = launch_pdl(span_count_kernel, dim3(gs), dim3(kSpanThreads), 0, st, order, rect, m2, co, n, tiles_x, tiles_y,
                 counts);
  if (e != cudaSuccess) return e;
  e = exclusive_scan<uint32_t, uint64_t>(counts, n, first, partials, out.num_instances, st);
  if (e != cudaSuccess) return e;
  // 3. Instances in depth order, into the buffer that makes the tile passes end in `out`.
  const int passes = radix_pass_count(plan.tile_bits);
  uint32_t* out_keys = out.tile_keys ? out.tile_keys : reinterpret_cast<uint32_t*>(ws + plan.off_ikeys[1]);
  uint32_t* ikeys[2];
  uint32_t* ivals[2];
  uint32_t* wk0 = reinterpret_cast<uint32_t*>(ws + plan.off_ikeys[0]);
  uint32_t* wv0 = reinterpret_cast<uint32_t*>(ws + plan.off_ivals);
  if (passes % 2 == 0) {
    ikeys[0] = out_keys; ivals[0] = out.point_list; ikeys[1] = wk0; ivals[1] = wv0;
  } else {
    ikeys[0] = wk0; ivals[0] = wv0; ikeys[1] = out_keys; ivals[1] = out.point_list;
  }
  const bool vec = ((reinterpret_cast<uintptr_t>(ikeys[0]) | reinterpret_cast<uintptr_t>(ivals[0])) & 15u) == 0;
  e = launch_pdl(span_emit_kernel, dim3(gs), dim3(kSpanThreads), 0, st, order, rect, m2, co, n, tiles_x, tiles_y,
                 (const uint64_t*)first, (const uint32_t*)counts, plan.capacity, ikeys[0], ivals[0], vec, passes,
                 radix_digit_width(plan.tile_bits), sort_t);
  if (e != cudaSuccess) return e;
  // 4. Stable sort by tile id; 5. tile ranges.
  radix_sort(ikeys, ivals, out.num_instances, 0, plan.capacity, plan.tile_bits, sort_t, err, true, st);
  {
    const unsigned gr = (unsigned)((plan.num_tiles + 7) / 8);  // 8 warps per block, one per tile
    e = launch_pdl(ranges_kernel, dim3(gr), dim3(256), 0, st, (const uint32_t*)out_keys,
                   (const int64_t*)out.num_instances, plan.capacity, (int)plan.num_tiles,
                   reinterpret_cast<uint2*>(out.ranges));
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

}  // namespace sdgs
