// Tile binning: the stable sort of the (tile << 32 | float32 depth bits) instance keys as an LSD
// sort in two digits, depth first, arranged so that neither digit's passes touch more data than
// they must.
//
// Depth digit: every instance of one Gaussian carries that Gaussian's depth, and instances are
// emitted in the order of the Gaussians.  So the depth passes of an LSD sort over the K instances
// give the same order as a stable radix sort of the n Gaussians by depth (ties keep ascending id)
// followed by emission in that order.  That sort runs over n keys, not K.
//
// Tile digit: instances exist only inside the per-row spans of tiles a Gaussian may reach
// (tile_reach.cuh).  For images of at most 256 tiles per side, the row spans themselves are
// emitted in depth order, sorted stably by row in one radix pass, and expanded into the tiles'
// lists per row (span binning, below).  Otherwise the instances, emitted in depth order, are
// radix-sorted stably by tile id (ceil(log2 tiles) bits, in passes of equal width <= 8 bits).
//
// Each radix pass is one kernel (digit histograms of all passes are accumulated while the keys are
// produced): a block ranks its tile of keys stably, finds the keys of each digit in earlier tiles
// by a decoupled look-back (bounded waits), and writes each digit's run contiguously.
#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "tile_reach.cuh"

namespace sdgs {

namespace {

constexpr int kRadixThreads = 256;
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
// Batches.  Every binning kernel takes the arguments of up to kMaxBatch independent problems by
// value (kernel parameter space, no device table) and serves problem blockIdx.y; a problem's
// blocks past its own grid size return at once.  One problem is a batch of one.
// ------------------------------------------------------------------------------------------
constexpr int kMaxBatch = kMaxBinBatch;

template <typename T>
struct Batch {
  T a[kMaxBatch];
};

template <typename T>
struct BatchLaunch {
  Batch<T> b;
  int count = 0;
  unsigned grid = 0;  // the largest grid of the batch's problems
  void add(const T& a) {
    b.a[count++] = a;
    grid = a.grid > grid ? a.grid : grid;
  }
};

template <typename K, typename T>
cudaError_t launch_batch(K kernel, const BatchLaunch<T>& L, unsigned threads, size_t smem, cudaStream_t st) {
  if (L.count == 0 || L.grid == 0) return cudaSuccess;
  return launch_pdl(kernel, dim3(L.grid, (unsigned)L.count), dim3(threads), smem, st, L.b);
}

// ------------------------------------------------------------------------------------------
// Device-wide exclusive scan: reduce per chunk, scan the chunk sums in one block, scan chunks.
// ------------------------------------------------------------------------------------------

template <typename TIn, typename TOut>
struct ScanArgs {
  const TIn* in;
  int64_t n;
  TOut* out;
  TOut* partials;
  int64_t* total_out;  // may be NULL
  unsigned grid;
};

template <typename TIn, typename TOut>
__global__ void __launch_bounds__(kScanThreads) scan_reduce_kernel(const Batch<ScanArgs<TIn, TOut>> b) {
  const ScanArgs<TIn, TOut>& a = b.a[blockIdx.y];
  if (blockIdx.x >= a.grid) return;
  griddep_wait();
  const int64_t base = (int64_t)blockIdx.x * kScanChunk;
  TOut sum = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const int64_t i = base + k * kScanThreads + threadIdx.x;
    if (i < a.n) sum += (TOut)a.in[i];
  }
  TOut total;
  block_inclusive_scan<TOut, kScanThreads>(sum, &total);
  if (threadIdx.x == 0) a.partials[blockIdx.x] = total;
}

template <typename TIn, typename TOut>
__global__ void __launch_bounds__(1024) scan_partials_kernel(const Batch<ScanArgs<TIn, TOut>> b) {
  const ScanArgs<TIn, TOut>& a = b.a[blockIdx.y];
  griddep_wait();
  const int64_t nb = (a.n + kScanChunk - 1) / kScanChunk;
  TOut carry = 0;
  for (int64_t base = 0; base < nb; base += 1024) {
    const int64_t i = base + threadIdx.x;
    const TOut x = i < nb ? a.partials[i] : TOut(0);
    TOut tot;
    const TOut incl = block_inclusive_scan<TOut, 1024>(x, &tot);
    if (i < nb) a.partials[i] = carry + incl - x;
    carry += tot;
  }
  if (threadIdx.x == 0 && a.total_out != nullptr) *a.total_out = (int64_t)carry;
}

template <typename TIn, typename TOut>
__global__ void __launch_bounds__(kScanThreads) scan_down_kernel(const Batch<ScanArgs<TIn, TOut>> b) {
  const ScanArgs<TIn, TOut>& a = b.a[blockIdx.y];
  if (blockIdx.x >= a.grid) return;
  griddep_wait();
  __shared__ TOut s[kScanChunk];
  const int64_t base = (int64_t)blockIdx.x * kScanChunk;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const int j = k * kScanThreads + threadIdx.x;
    s[j] = (base + j < a.n) ? (TOut)a.in[base + j] : TOut(0);
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
  const TOut off = a.partials[blockIdx.x] + incl - local;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) s[threadIdx.x * kScanItems + k] = off + v[k];
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const int j = k * kScanThreads + threadIdx.x;
    if (base + j < a.n) a.out[base + j] = s[j];
  }
}

// The whole scan in one block, for up to kSingleScanItems * 1024 elements: the block stages the
// input in shared memory with coalesced loads, each thread sums its run of consecutive elements,
// the block scans the sums, and each thread writes its run.
constexpr int kSingleScanItems = 11;

template <typename TIn, typename TOut>
__global__ void __launch_bounds__(1024) scan_single_kernel(const Batch<ScanArgs<TIn, TOut>> b) {
  const ScanArgs<TIn, TOut>& a = b.a[blockIdx.y];
  __shared__ TIn s_in[kSingleScanItems * 1024];
  griddep_wait();
  const int n = (int)a.n;  // <= kSingleScanItems * 1024
  {
    TIn v[kSingleScanItems];  // every load in flight before any is used
#pragma unroll
    for (int k = 0; k < kSingleScanItems; ++k) {
      const int i = k * 1024 + threadIdx.x;
      v[k] = i < n ? a.in[i] : TIn(0);
    }
#pragma unroll
    for (int k = 0; k < kSingleScanItems; ++k) {
      const int i = k * 1024 + threadIdx.x;
      if (i < n) s_in[i] = v[k];
    }
  }
  __syncthreads();
  const int per = (n + 1023) / 1024;  // <= kSingleScanItems
  const int base = threadIdx.x * per;
  TOut local = 0;
#pragma unroll
  for (int k = 0; k < kSingleScanItems; ++k)
    if (k < per && base + k < n) local += (TOut)s_in[base + k];
  TOut tot;
  TOut run = block_inclusive_scan<TOut, 1024>(local, &tot) - local;
#pragma unroll
  for (int k = 0; k < kSingleScanItems; ++k) {
    if (k < per && base + k < n) {
      const TOut v = (TOut)s_in[base + k];
      a.out[base + k] = run;
      run += v;
    }
  }
  if (threadIdx.x == 0 && a.total_out != nullptr) *a.total_out = (int64_t)tot;
}

// Exclusive scans of a batch of arrays (one problem each, in[i] -> out[i], total in *total_out).
template <typename TIn, typename TOut>
cudaError_t exclusive_scan(const ScanArgs<TIn, TOut>* jobs, int count, cudaStream_t st) {
  BatchLaunch<ScanArgs<TIn, TOut>> small, big;
  for (int j = 0; j < count; ++j) {
    ScanArgs<TIn, TOut> a = jobs[j];
    if (a.n <= (int64_t)kSingleScanItems * 1024) {
      a.grid = 1;
      small.add(a);
    } else {
      a.grid = (unsigned)((a.n + kScanChunk - 1) / kScanChunk);
      big.add(a);
    }
  }
  cudaError_t e = launch_batch(scan_single_kernel<TIn, TOut>, small, 1024, 0, st);
  if (e == cudaSuccess) e = launch_batch(scan_reduce_kernel<TIn, TOut>, big, kScanThreads, 0, st);
  if (e == cudaSuccess && big.count > 0) {
    BatchLaunch<ScanArgs<TIn, TOut>> one = big;
    one.grid = 1;
    e = launch_batch(scan_partials_kernel<TIn, TOut>, one, 1024, 0, st);
  }
  if (e == cudaSuccess) e = launch_batch(scan_down_kernel<TIn, TOut>, big, kScanThreads, 0, st);
  return e;
}

template <typename TIn, typename TOut>
cudaError_t exclusive_scan(const TIn* in, int64_t n, TOut* out, uint64_t* partials, int64_t* total_out,
                           cudaStream_t st) {
  const ScanArgs<TIn, TOut> a{in, n, out, reinterpret_cast<TOut*>(partials), total_out, 0};
  return exclusive_scan(&a, 1, st);
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
__device__ __forceinline__ void load_and_rank(const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
                                              int64_t wbase, int64_t n, int shift, int width, uint32_t* whist,
                                              uint32_t key[ITEMS], uint32_t val[ITEMS], uint32_t rank[ITEMS]) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = lanemask_lt();
  const uint32_t dmask = (1u << width) - 1u;
#pragma unroll
  for (int r = 0; r < ITEMS; ++r) {
    const int64_t idx = wbase + r * 32 + lane;
    key[r] = (FULL || idx < n) ? keys_in[idx] : 0u;
    val[r] = (FULL || idx < n) ? vals_in[idx] : 0u;
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

// Keys with digit dg in sort tiles 0 .. tile - 1, from the status words of the earlier tiles: each
// round loads the next kLookbackWindow of them at once (nearest first) and adds their counts up to
// the first inclusive one; an entry not yet published ends the round, and the next round starts at
// it after a short sleep.  Every wait is bounded: after spin_limit rounds that found an
// unpublished entry the block sets this pass's bit of *err and returns what it has.
__device__ __forceinline__ uint32_t lookback(const uint32_t* status, int64_t tile, int dg, int spin_limit,
                                             uint32_t pass_bit, uint32_t* err) {
  uint32_t before = 0;
  int64_t j = tile - 1;
  int spins = 0;
  while (j >= 0) {
    uint32_t st[kLookbackWindow];
#pragma unroll
    for (int w = 0; w < kLookbackWindow; ++w)
      st[w] = j - w >= 0 ? load_status(status + (j - w) * kBins + dg) : kStatusInclusive;  // before tile 0: 0
    bool done = false, blocked = false;
#pragma unroll
    for (int w = 0; w < kLookbackWindow; ++w) {
      if (done || blocked) continue;
      if ((st[w] & ~kStatusCount) == 0u) {
        blocked = true;  // not published yet: poll it next round
        continue;
      }
      before += st[w] & kStatusCount;
      if (st[w] & kStatusInclusive) done = true;
      else --j;
    }
    if (done) break;
    if (blocked) {
      if (++spins > spin_limit) {
        atomicOr(err, pass_bit);
        break;
      }
      __nanosleep(32);
    }
  }
  return before;
}

// One radix pass of one problem (keys_in, vals_in -> keys_out, vals_out by the digit at shift).
struct PassArgs {
  const uint32_t* keys_in;
  const uint32_t* vals_in;
  uint32_t* keys_out;
  uint32_t* vals_out;
  const int64_t* nptr;  // element count on the device (clipped to cap), or NULL for n_static
  int64_t n_static, cap;
  int shift, width;
  const uint32_t* digit_hist;
  uint32_t* status;
  uint32_t* ticket;
  uint32_t* err;
  uint32_t pass_bit;
  int spin_limit;
  unsigned grid;
};

// THREADS threads with ITEMS keys each; threads past the kBins digits sit out the digit phases.
template <int ITEMS, int THREADS = kRadixThreads>
__global__ void __launch_bounds__(THREADS, THREADS > kRadixThreads ? 1024 / THREADS : (ITEMS >= 12 ? 4 : 5))
    onesweep_kernel(const Batch<PassArgs> batch) {
  const PassArgs& pa = batch.a[blockIdx.y];
  if (blockIdx.x >= pa.grid) return;
  const uint32_t* __restrict__ keys_in = pa.keys_in;
  const uint32_t* __restrict__ vals_in = pa.vals_in;
  uint32_t* __restrict__ keys_out = pa.keys_out;
  uint32_t* __restrict__ vals_out = pa.vals_out;
  const int64_t* nptr = pa.nptr;
  const int64_t n_static = pa.n_static, cap = pa.cap;
  const int shift = pa.shift, width = pa.width;
  const uint32_t* __restrict__ digit_hist = pa.digit_hist;
  uint32_t* status = pa.status;
  uint32_t* ticket = pa.ticket;
  uint32_t* err = pa.err;
  const uint32_t pass_bit = pa.pass_bit;
  const int spin_limit = pa.spin_limit;
  griddep_wait();
  constexpr int TILE = THREADS * ITEMS;
  constexpr int WARPS = THREADS / 32;
  static_assert(THREADS >= kBins, "one thread per digit");
  __shared__ uint32_t s_keys[TILE];
  __shared__ uint32_t s_vals[TILE];
  __shared__ uint32_t s_whist[WARPS][kBins];
  __shared__ uint32_t s_dstart[kBins];
  __shared__ uint32_t s_gbase[kBins];
  __shared__ uint32_t s_tile;
  if (threadIdx.x == 0) s_tile = atomicAdd(ticket, 1u);
  for (int i = threadIdx.x; i < WARPS * kBins; i += THREADS) (&s_whist[0][0])[i] = 0;
  __syncthreads();
  const int64_t tile = s_tile;
  const int64_t n = element_count(nptr, n_static, cap);
  const int64_t base = tile * TILE;
  if (base >= n) return;  // so do all later tiles: nobody waits on this one
  // An earlier pass gave up waiting: its output is not a permutation of its input, so this pass's
  // digit histogram no longer bounds its positions.  Skip (ranges_kernel then empties the lists).
  // (Bits of this pass are set only by its own blocks, which never make another block skip.)
  if ((*reinterpret_cast<volatile uint32_t*>(err) & (pass_bit - 1u)) != 0u) return;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t dmask = (1u << width) - 1u;
  const int64_t wbase = base + (int64_t)warp * 32 * ITEMS;
  const bool full = base + TILE <= n;  // uniform over the block
  const int dg = threadIdx.x;
  const bool digit = dg < kBins;       // this thread owns bin dg
  const bool used = dg <= (int)dmask;  // digits of `width` bits: the other bins stay empty
  uint32_t* mine = status + tile * kBins + dg;
  uint32_t run = 0;  // this tile's keys with digit dg
  {
    uint32_t key[ITEMS], val[ITEMS], rank[ITEMS];
    if (full) load_and_rank<ITEMS, true>(keys_in, vals_in, wbase, n, shift, width, s_whist[warp], key, val, rank);
    else load_and_rank<ITEMS, false>(keys_in, vals_in, wbase, n, shift, width, s_whist[warp], key, val, rank);
    __syncthreads();
    if (digit) {
#pragma unroll
      for (int w = 0; w < WARPS; ++w) {
        const uint32_t c = s_whist[w][dg];
        s_whist[w][dg] = run;
        run += c;
      }
    }
    // publish this tile's count at once, so later tiles can pass over it while it waits
    if (used) store_status(mine, (tile == 0 ? kStatusInclusive : kStatusAggregate) | run);
    uint32_t tot;
    const uint32_t incl = block_inclusive_scan<uint32_t, THREADS>(run, &tot);
    if (digit) s_dstart[dg] = incl - run;
    __syncthreads();
    // the tile's keys in digit order, in shared memory (stable: warps, then ranks)
#pragma unroll
    for (int r = 0; r < ITEMS; ++r) {
      const int64_t idx = wbase + r * 32 + lane;
      if (full || idx < n) {
        const uint32_t d = (key[r] >> shift) & dmask;
        const uint32_t pos = s_dstart[d] + s_whist[warp][d] + rank[r];
        s_keys[pos] = key[r];
        s_vals[pos] = val[r];
      }
    }
  }
  const uint32_t before = used && tile > 0 ? lookback(status, tile, dg, spin_limit, pass_bit, err) : 0u;
  if (used && tile > 0) store_status(mine, kStatusInclusive | (before + run));
  {
    uint32_t tot;
    const uint32_t all = digit ? digit_hist[dg] : 0u;
    const uint32_t gincl = block_inclusive_scan<uint32_t, THREADS>(all, &tot);
    if (digit) s_gbase[dg] = gincl - all + before;
  }
  __syncthreads();
  if (full) {
#pragma unroll
    for (int r = 0; r < ITEMS; ++r) {
      const int i = r * THREADS + threadIdx.x;
      const uint32_t k = s_keys[i];
      const uint32_t d = (k >> shift) & dmask;
      const uint32_t g = s_gbase[d] + (uint32_t)i - s_dstart[d];
      if (g < (uint64_t)n) {  // always, unless a look-back gave up
        keys_out[g] = k;
        vals_out[g] = s_vals[i];
      }
    }
  } else {
    const int cnt = (int)(n - base);
    for (int i = threadIdx.x; i < cnt; i += THREADS) {
      const uint32_t k = s_keys[i];
      const uint32_t d = (k >> shift) & dmask;
      const uint32_t g = s_gbase[d] + (uint32_t)i - s_dstart[d];
      if (g < (uint64_t)n) {
        keys_out[g] = k;
        vals_out[g] = s_vals[i];
      }
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

// Tile size of a sort of `cap` slots, in keys per kRadixThreads threads: 12 (3072-key tiles, run
// as 256 threads x 12) when that still gives two blocks per SM, else 8 (2048-key tiles, run as
// 512 threads x 4).  Fewer, larger tiles shorten the look-back chains of small sorts (a 300k-key
// depth pass: 147 tiles of 2048 keys run faster than 293 of 1024).
int sort_items(int64_t cap) {
  const int64_t want = 2 * (int64_t)device_sm_count();
  if ((cap + 12 * kRadixThreads - 1) / (12 * kRadixThreads) >= want) return 12;
  return 8;
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
// One radix sort (keys, vals ping-pong) of a batch of problems.
struct SortJob {
  uint32_t* keys[2];
  uint32_t* vals[2];
  const int64_t* nptr;
  int64_t n_static, cap;
  int bits;
  uint32_t* scratch;  // sort_scratch_bytes(cap, bits)
  uint32_t* err;
  int first_pass;     // the error bit of pass p is 1 << (first_pass + p)
};

// Sorts every job by bits [0, bits) in ceil(bits / 8) passes of equal digit width, ping-ponging
// between buffers 0 and 1 (a job whose passes are over sits out the later launches); returns in
// cur[j] the buffer holding job j's result.  With hist_ready the caller has cleared the scratch
// (sort_clear) and accumulated the digit histograms of all keys into its first kMaxPasses * kBins
// words while producing them.
cudaError_t radix_sort(const SortJob* jobs, int count, bool hist_ready, cudaStream_t st, int* cur,
                       int spin_limit = kLookbackSpins) {
  int max_passes = 0;
  for (int j = 0; j < count; ++j) {
    cur[j] = 0;
    if (jobs[j].cap > 0 && jobs[j].bits > 0) max_passes = std::max(max_passes, radix_pass_count(jobs[j].bits));
  }
  cudaError_t e = cudaSuccess;
  if (!hist_ready) {  // (single jobs only: the test support path)
    for (int j = 0; j < count && e == cudaSuccess; ++j) {
      const SortJob& J = jobs[j];
      if (J.cap <= 0 || J.bits <= 0) continue;
      sort_clear(J.scratch, J.cap, J.bits, st);
      const int64_t hist_blocks = std::min<int64_t>((J.cap + kRadixThreads - 1) / kRadixThreads, 4 * device_sm_count());
      digit_hist_kernel<<<(unsigned)hist_blocks, kRadixThreads, 0, st>>>(J.keys[0], J.nptr, J.n_static, J.cap,
                                                                         radix_pass_count(J.bits),
                                                                         radix_digit_width(J.bits), J.scratch);
      e = cudaGetLastError();
    }
  }
  for (int p = 0; p < max_passes && e == cudaSuccess; ++p) {
    BatchLaunch<PassArgs> l12, l8;  // the two tile sizes launch separately
    for (int j = 0; j < count; ++j) {
      const SortJob& J = jobs[j];
      if (J.cap <= 0 || J.bits <= 0 || p >= radix_pass_count(J.bits)) continue;
      const int width = radix_digit_width(J.bits);
      const int64_t nblocks = sort_blocks(J.cap);
      uint32_t* hist = J.scratch;
      uint32_t* tickets = hist + kMaxPasses * kBins;
      uint32_t* status = tickets + kMaxPasses;
      PassArgs a;
      a.keys_in = J.keys[cur[j]]; a.vals_in = J.vals[cur[j]];
      a.keys_out = J.keys[cur[j] ^ 1]; a.vals_out = J.vals[cur[j] ^ 1];
      a.nptr = J.nptr; a.n_static = J.n_static; a.cap = J.cap;
      a.shift = p * width; a.width = width;
      a.digit_hist = hist + p * kBins;
      a.status = status + (size_t)p * nblocks * kBins;
      a.ticket = tickets + p;
      a.err = J.err;
      a.pass_bit = 1u << (J.first_pass + p);
      a.spin_limit = spin_limit;
      a.grid = (unsigned)nblocks;
      (sort_items(J.cap) == 12 ? l12 : l8).add(a);
      cur[j] ^= 1;
    }
    // (the 2048-key tiles run as 512 threads with 4 keys each: twice the warps of 256 x 8 to hide
    // the latency of the pass's dependent phases, the same tiles and look-back chain)
    e = launch_batch(onesweep_kernel<12>, l12, kRadixThreads, 0, st);
    if (e == cudaSuccess) e = launch_batch(onesweep_kernel<4, 2 * kRadixThreads>, l8, 2 * kRadixThreads, 0, st);
  }
  return e;
}

// ------------------------------------------------------------------------------------------
// Binning-specific kernels.
// ------------------------------------------------------------------------------------------

// Zeroes the words binning accumulates into or reads before writing: the error word, the tile
// ranges and the instance count (when there are no Gaussians) and both sorts' scratch.  One kernel
// instead of several memsets keeps the render's launches a chain of kernels.
struct ClearJob {
  static constexpr int kSlots = 7;
  uint32_t* ptr[kSlots];
  size_t words[kSlots];
  unsigned grid;
};

__global__ void __launch_bounds__(256) clear_kernel(const Batch<ClearJob> b) {
  const ClearJob& job = b.a[blockIdx.y];
  if (blockIdx.x >= job.grid) return;
  griddep_wait();
  const size_t stride = (size_t)job.grid * blockDim.x;
  for (int k = 0; k < ClearJob::kSlots; ++k) {
    uint32_t* p = job.ptr[k];
    if (p == nullptr) continue;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < job.words[k]; i += stride) p[i] = 0u;
  }
}

// Depth keys of the Gaussians (culled ones last) and their digit histograms for the depth sort.  A
// few blocks per SM stride over the Gaussians, so that few block histograms are added globally.
struct DepthKeysArgs {
  const float* depth;
  const ushort4* rect;
  int64_t n;
  uint32_t* keys;
  uint32_t* vals;
  uint32_t* hist;
  uint32_t* visible;  // visible Gaussians are added up here, or NULL
  unsigned grid;
};

__global__ void __launch_bounds__(kRadixThreads) depth_keys_kernel(const Batch<DepthKeysArgs> b) {
  const DepthKeysArgs& a = b.a[blockIdx.y];
  if (blockIdx.x >= a.grid) return;
  const float* __restrict__ depth = a.depth;
  const ushort4* __restrict__ rect = a.rect;
  const int64_t n = a.n;
  uint32_t* __restrict__ keys = a.keys;
  uint32_t* __restrict__ vals = a.vals;
  uint32_t* __restrict__ hist = a.hist;
  griddep_wait();
  __shared__ uint32_t s_hist[kMaxPasses][kBins];
  __shared__ uint32_t s_vis;
  for (int i = threadIdx.x; i < kMaxPasses * kBins; i += kRadixThreads) (&s_hist[0][0])[i] = 0;
  if (threadIdx.x == 0) s_vis = 0;
  __syncthreads();
  uint32_t nvis = 0;
  constexpr int U = 4;  // elements per thread per round, their loads issued together
  const int64_t stride = (int64_t)a.grid * kRadixThreads * U;
  for (int64_t i0 = (int64_t)blockIdx.x * kRadixThreads * U; i0 < n; i0 += stride) {  // uniform over the block
    ushort4 r[U];
    float z[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = i0 + u * kRadixThreads + threadIdx.x;
      r[u] = i < n ? rect[i] : make_ushort4(0, 0, 0, 0);
      z[u] = i < n ? depth[i] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = i0 + u * kRadixThreads + threadIdx.x;
      uint32_t k = 0;
      if (i < n) {
        const bool vis = r[u].z > r[u].x && r[u].w > r[u].y;
        k = vis ? __float_as_uint(z[u]) : 0xffffffffu;  // visible depths are positive
        nvis += vis ? 1u : 0u;
        keys[i] = k;
        vals[i] = (uint32_t)i;
      }
      count_digits(s_hist, k, i < n, 4, 8);
    }
  }
  if (a.visible != nullptr) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nvis += __shfl_xor_sync(0xffffffffu, nvis, o);
    if ((threadIdx.x & 31) == 0 && nvis) atomicAdd(&s_vis, nvis);
  }
  __syncthreads();
  flush_digits(s_hist, 4, hist);
  if (a.visible != nullptr && threadIdx.x == 0 && s_vis) atomicAdd(a.visible, s_vis);
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

// Span walks.  A warp takes 32 consecutive depth-ordered Gaussians and flattens their rows: lane i
// sets up Gaussian i (its rectangle, clipped to the grid, and its reachability rule, kept in
// shared memory), then the warp walks the sequence of (Gaussian, row) pairs 32 rows at a time, one
// row per lane, so that no lane idles behind a Gaussian with many rows.
constexpr int kWalkThreads = 256;
constexpr int kWalkWarps = kWalkThreads / 32;

struct WalkWarp {  // one warp's 32 Gaussians, structure of arrays (conflict-free by owner lane)
  float u[32], v[32], a[32], b[32], det[32], aQ[32], reach_y[32], dyr[32], padx[32];
  int mode[32], rx0[32], rx1[32], y0[32];
  uint32_t g[32];
};

// Sets up this lane's Gaussian (depth-order position s) and returns its number of candidate rows;
// the warp's row sequence is then given by the inclusive scan of the counts.
__device__ __forceinline__ int walk_setup(WalkWarp& w, const uint32_t* __restrict__ order,
                                          const ushort4* __restrict__ rect, const float2* __restrict__ mean2d,
                                          const float4* __restrict__ conic_opacity, int64_t s, int64_t n,
                                          int tiles_x, int tiles_y) {
  const int lane = threadIdx.x & 31;
  int nr = 0;
  if (s < n) {
    const uint32_t g = order[s];
    const ushort4 r = clip_rect(rect[g], tiles_x, tiles_y);
    if (r.z > r.x && r.w > r.y) {
      const SpanRule q = span_setup(mean2d[g], conic_opacity[g]);
      int y0, y1;
      span_rows(q, r.y, r.w, &y0, &y1);
      nr = y1 - y0;
      w.u[lane] = q.u; w.v[lane] = q.v; w.a[lane] = q.a; w.b[lane] = q.b; w.det[lane] = q.det;
      w.aQ[lane] = q.aQ; w.reach_y[lane] = q.reach_y; w.dyr[lane] = q.dyr; w.padx[lane] = q.padx;
      w.mode[lane] = q.mode; w.rx0[lane] = r.x; w.rx1[lane] = r.z; w.y0[lane] = y0; w.g[lane] = g;
    }
  }
  __syncwarp();
  return nr;
}

// The lane holding element k of a sequence whose lanes own runs of lengths given by their
// inclusive prefix `incl` (the first lane with incl > k); k < the total.  All lanes call.
__device__ __forceinline__ int owner_lane(uint32_t incl, uint32_t k) {
  int o = 0;
#pragma unroll
  for (int step = 16; step >= 1; step >>= 1) {
    const uint32_t v = __shfl_sync(0xffffffffu, incl, o + step - 1);
    if (v <= k) o += step;
  }
  return o;
}

// Kept tiles [*x0, *x1) of row k of the warp's row sequence (row_incl: inclusive row counts by
// lane); *ty its tile row, *o its Gaussian's lane.
__device__ __forceinline__ void walk_row(const WalkWarp& w, uint32_t row_incl, int nr, uint32_t k, int* o, int* ty,
                                         int* x0, int* x1) {
  *o = owner_lane(row_incl, k);
  const uint32_t first_row = __shfl_sync(0xffffffffu, row_incl - (uint32_t)nr, *o);
  const int i = *o;
  SpanRule q;
  q.u = w.u[i]; q.v = w.v[i]; q.a = w.a[i]; q.b = w.b[i]; q.det = w.det[i]; q.aQ = w.aQ[i];
  q.hx = 0.f; q.reach_y = w.reach_y[i]; q.dyr = w.dyr[i]; q.padx = w.padx[i]; q.mode = w.mode[i];
  *ty = w.y0[i] + (int)(k - first_row);
  span_cols(q, *ty, w.rx0[i], w.rx1[i], x0, x1);
}

// Kept-tile count of each warp's 32 depth-ordered Gaussians (wcount[warp]).
// Arguments of the span walks of one problem.
struct WalkArgs {
  const uint32_t* order;  // depth-ordered Gaussian ids
  const ushort4* rect;
  const float2* mean2d;
  const float4* conic_opacity;
  int64_t n;
  int tiles_x, tiles_y;
  const uint32_t* err;
  uint32_t* wcount;       // count walk: kept tiles per warp chunk
  const uint64_t* wfirst; // emit: first instance of each warp chunk
  int64_t cap;
  uint32_t* keys;
  uint32_t* vals;
  int passes, width;      // tile-digit passes whose histograms the emit accumulates into hist
  uint32_t* hist;
  unsigned grid;
};

__global__ void __launch_bounds__(kWalkThreads) walk_count_kernel(const Batch<WalkArgs> b) {
  const WalkArgs& A = b.a[blockIdx.y];
  if (blockIdx.x >= A.grid) return;
  const uint32_t* __restrict__ order = A.order;
  const ushort4* __restrict__ rect = A.rect;
  const float2* __restrict__ mean2d = A.mean2d;
  const float4* __restrict__ conic_opacity = A.conic_opacity;
  const int64_t n = A.n;
  const int tiles_x = A.tiles_x, tiles_y = A.tiles_y;
  const uint32_t* err = A.err;
  uint32_t* __restrict__ wcount = A.wcount;
  griddep_wait();
  __shared__ WalkWarp s_walk[kWalkWarps];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t wg = (int64_t)blockIdx.x * kWalkWarps + warp;
  if (wg * 32 >= n) return;  // whole warps
  if (*err != 0u) {  // the depth sort gave up: `order` may hold any value, so emit nothing
    if (lane == 0) wcount[wg] = 0;
    return;
  }
  WalkWarp& w = s_walk[warp];
  const int nr = walk_setup(w, order, rect, mean2d, conic_opacity, wg * 32 + lane, n, tiles_x, tiles_y);
  const uint32_t row_incl = warp_inclusive_scan((uint32_t)nr);
  const uint32_t rows = __shfl_sync(0xffffffffu, row_incl, 31);
  uint32_t sum = 0;
  for (uint32_t rb = 0; rb < rows; rb += 32) {
    const uint32_t k = rb + lane;
    int o, ty, x0, x1;
    walk_row(w, row_incl, nr, k < rows ? k : rows - 1, &o, &ty, &x0, &x1);
    if (k < rows) sum += (uint32_t)(x1 - x0);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, off);
  if (lane == 0) wcount[wg] = sum;
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

// Writes the (tile id, Gaussian id) pairs of each warp's 32 depth-ordered Gaussians from the warp's
// first instance wfirst[warp], row-major over each Gaussian's spans, and accumulates the tile-digit
// histograms of what it writes.  The warp walks its row sequence 32 rows at a time (one row per
// lane, as in walk_count_kernel); a warp scan places the rows' spans, and the lanes then store the
// chunk's instances 32 consecutive ones at a time (coalesced).  Positions >= cap are dropped.
__global__ void __launch_bounds__(kWalkThreads) walk_emit_kernel(const Batch<WalkArgs> b) {
  const WalkArgs& A = b.a[blockIdx.y];
  if (blockIdx.x >= A.grid) return;
  const uint32_t* __restrict__ order = A.order;
  const ushort4* __restrict__ rect = A.rect;
  const float2* __restrict__ mean2d = A.mean2d;
  const float4* __restrict__ conic_opacity = A.conic_opacity;
  const int64_t n = A.n;
  const int tiles_x = A.tiles_x, tiles_y = A.tiles_y;
  const uint64_t* __restrict__ wfirst = A.wfirst;
  const int64_t cap = A.cap;
  uint32_t* __restrict__ keys = A.keys;
  uint32_t* __restrict__ vals = A.vals;
  const int passes = A.passes, width = A.width;
  const uint32_t* err = A.err;
  uint32_t* __restrict__ hist = A.hist;
  griddep_wait();
  __shared__ WalkWarp s_walk[kWalkWarps];
  __shared__ uint32_t s_hist[kMaxPasses][kBins];
  __shared__ int32_t s_diff0[kBins + 1];
  __shared__ uint32_t s_all0;
  for (int i = threadIdx.x; i < kMaxPasses * kBins; i += kWalkThreads) (&s_hist[0][0])[i] = 0;
  for (int i = threadIdx.x; i <= kBins; i += kWalkThreads) s_diff0[i] = 0;
  if (threadIdx.x == 0) s_all0 = 0;
  __syncthreads();
  const DigitAcc acc{s_hist, s_diff0, &s_all0};
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t wg = (int64_t)blockIdx.x * kWalkWarps + warp;
  if (wg * 32 < n && *err == 0u) {  // uniform over the warp
    WalkWarp& w = s_walk[warp];
    const int nr = walk_setup(w, order, rect, mean2d, conic_opacity, wg * 32 + lane, n, tiles_x, tiles_y);
    const uint32_t row_incl = warp_inclusive_scan((uint32_t)nr);
    const uint32_t rows = __shfl_sync(0xffffffffu, row_incl, 31);
    uint64_t pos = wfirst[wg];
    for (uint32_t rb = 0; rb < rows && pos < (uint64_t)cap; rb += 32) {  // uniform
      const uint32_t k = rb + lane;
      int o, ty, x0, x1;
      walk_row(w, row_incl, nr, k < rows ? k : rows - 1, &o, &ty, &x0, &x1);
      const uint32_t len = k < rows ? (uint32_t)(x1 - x0) : 0u;
      const uint32_t incl = warp_inclusive_scan(len);
      const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
      const uint32_t id0 = (uint32_t)ty * (uint32_t)tiles_x + (uint32_t)x0;  // the row's first tile id
      const uint32_t gid = w.g[o];
      {  // digit histograms of the instances this row writes
        const int64_t room = cap - ((int64_t)pos + (int64_t)(incl - len));
        const uint32_t written = room <= 0 ? 0u : (room < (int64_t)len ? (uint32_t)room : len);
        count_span_digits(acc, id0, written, passes, width);
      }
      for (uint32_t j0 = 0; j0 < total; j0 += 32) {
        const uint32_t j = j0 + lane;
        const int rl = owner_lane(incl, j < total ? j : total - 1);  // the row holding instance j
        const uint32_t r_excl = __shfl_sync(0xffffffffu, incl - len, rl);
        const uint32_t r_id0 = __shfl_sync(0xffffffffu, id0, rl);
        const uint32_t r_gid = __shfl_sync(0xffffffffu, gid, rl);
        const uint64_t p = pos + j;
        if (j < total && p < (uint64_t)cap) {
          keys[p] = r_id0 + (j - r_excl);
          vals[p] = r_gid;
        }
      }
      pos += total;
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

// ------------------------------------------------------------------------------------------
// Span binning (images of at most kSpanMaxTiles tiles per side).  Instead of one record per
// (tile, Gaussian) instance, the emit walk writes one record per kept row span of a Gaussian, in
// depth order: key = row | x0 << 8 | (len - 1) << 16, value = Gaussian id.  One stable radix
// pass over the row puts each row's spans together (still in depth order), and the expansion then
// writes every span's instances into its tiles' lists: each chunk of a row's spans counts its
// instances per column (span_count_kernel), and each chunk then finds where its instances go from
// those counts, places them in (column, depth) order through shared memory and writes every
// column's run contiguously (span_expand_kernel).  The lists, ranges and instance count are those of the
// instance path: the tile sort is stable, so a tile's list is its instances in depth order.
// ------------------------------------------------------------------------------------------
constexpr int kSpanMaxTiles = 256;   // tiles per side: row and x0 fit 8 bits, len - 1 16 bits
constexpr int kSpanThreads = 256;
constexpr int kSpanPer = 4;          // spans per thread per expansion chunk, at most
constexpr int kSpanWindow = 8192;    // instances a chunk stages in shared memory

__device__ __forceinline__ uint32_t span_key(int row, int x0, int len) {
  return (uint32_t)row | ((uint32_t)x0 << 8) | ((uint32_t)(len - 1) << 16);
}
__device__ __forceinline__ int span_x0(uint32_t k) { return (int)((k >> 8) & 0xffu); }
__device__ __forceinline__ int span_len(uint32_t k) { return (int)(k >> 16) + 1; }

// Single-pass span emit: the count walk, the scan of its totals and the emit in one kernel.  Each
// block (8 warps, 256 depth-ordered Gaussians, numbered by a ticket taken when it starts) walks its
// warps' rows once, keeping up to kWalkKeep spans per warp in shared memory, and publishes its
// span and instance totals at once; a decoupled look-back over the earlier blocks' totals (32 per
// round, one per lane) gives its first span and first instance, and it then writes its spans,
// cutting them at cap (a span whose first instance lies at depth-order position >= cap is dropped,
// one that crosses cap is cut there).  A warp with more spans than it kept walks its
// rows again while writing.  The last block to finish sets the kept span count.  Every wait is
// bounded: a block that gives up sets pass_bit in *err (the row sort then skips and the lists
// stay empty).
constexpr int kWalkKeep = 224;                          // spans per warp kept between walk and write
constexpr uint64_t kWalkAggregate = 1ull << 62;         // the block's own totals
constexpr uint64_t kWalkInclusive = 2ull << 62;         // totals of blocks 0 .. this one
constexpr uint64_t kWalkField = (1ull << 31) - 1;       // 31-bit fields: instances << 31 | spans

__device__ __forceinline__ uint64_t walk_pack(uint64_t spans, uint64_t inst) {
  return (min(inst, kWalkField) << 31) | min(spans, kWalkField);
}

struct SpanWalkArgs {
  const uint32_t* order;  // depth-ordered Gaussian ids
  const ushort4* rect;
  const float2* mean2d;
  const float4* conic_opacity;
  int64_t n;
  int tiles_x, tiles_y;
  uint32_t* err;
  uint32_t pass_bit;
  int spin_limit;
  int64_t cap;
  uint32_t* keys;             // spans out (depth order)
  uint32_t* vals;
  uint32_t* hist;             // row histogram (the row sort's digit histogram)
  int64_t* num_instances;     // K (zeroed before binning)
  uint32_t* counters;         // [0] ticket, [1] blocks done, [2..3] ~(first dropped span), [4] visible
                              // Gaussians (from the depth keys), [6..7] spans kept (int64); zeroed first
  uint64_t* status;           // [grid] (zeroed)
  unsigned grid;
};

__global__ void __launch_bounds__(kWalkThreads) span_walk_kernel(const Batch<SpanWalkArgs> b) {
  const SpanWalkArgs& A = b.a[blockIdx.y];
  if (blockIdx.x >= A.grid) return;
  griddep_wait();
  __shared__ WalkWarp s_walk[kWalkWarps];
  __shared__ uint32_t s_key[kWalkWarps][kWalkKeep];
  __shared__ uint32_t s_gid[kWalkWarps][kWalkKeep];
  __shared__ uint32_t s_ioff[kWalkWarps][kWalkKeep];
  __shared__ uint32_t s_rows[kSpanMaxTiles];
  __shared__ uint32_t s_wsp[kWalkWarps], s_win[kWalkWarps];
  __shared__ uint64_t s_before_sp, s_before_in;
  __shared__ uint32_t s_tile;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned lt = lanemask_lt();
  if (threadIdx.x == 0) s_tile = atomicAdd(&A.counters[0], 1u);
  for (int i = threadIdx.x; i < kSpanMaxTiles; i += kWalkThreads) s_rows[i] = 0;
  __syncthreads();
  const int64_t tile = s_tile;
  // Culled Gaussians come last in depth order: the blocks past the visible ones have nothing to
  // write and nobody waits on them.
  const int64_t blocks = ((int64_t)A.counters[4] + kWalkThreads - 1) / kWalkThreads;
  if (tile >= blocks) return;
  const bool live = *reinterpret_cast<volatile uint32_t*>(A.err) == 0u;  // the depth sort completed
  // 1. walk: count this warp's spans and instances, keeping the first kWalkKeep spans
  const int64_t wg = tile * kWalkWarps + warp;
  WalkWarp& w = s_walk[warp];
  int nr = 0;
  uint32_t row_incl = 0, rows = 0, nsp = 0, ninst = 0;
  if (live && wg * 32 < A.n) {  // uniform over the warp
    nr = walk_setup(w, A.order, A.rect, A.mean2d, A.conic_opacity, wg * 32 + lane, A.n, A.tiles_x, A.tiles_y);
    row_incl = warp_inclusive_scan((uint32_t)nr);
    rows = __shfl_sync(0xffffffffu, row_incl, 31);
    for (uint32_t rb = 0; rb < rows; rb += 32) {
      const uint32_t k = rb + lane;
      int o, ty, x0, x1;
      walk_row(w, row_incl, nr, k < rows ? k : rows - 1, &o, &ty, &x0, &x1);
      const uint32_t len = k < rows ? (uint32_t)(x1 - x0) : 0u;
      const uint32_t incl = warp_inclusive_scan(len);
      const unsigned has = __ballot_sync(0xffffffffu, len > 0u);
      if (len > 0u) {
        const uint32_t j = nsp + (uint32_t)__popc(has & lt);
        if (j < (uint32_t)kWalkKeep) {
          s_key[warp][j] = span_key(ty, x0, (int)len);
          s_gid[warp][j] = w.g[o];
          s_ioff[warp][j] = ninst + (incl - len);
        }
      }
      nsp += (uint32_t)__popc(has);
      ninst += __shfl_sync(0xffffffffu, incl, 31);
    }
  }
  if (lane == 0) {
    s_wsp[warp] = nsp;
    s_win[warp] = ninst;
  }
  __syncthreads();
  // 2. block totals (warp prefixes), published at once; then the look-back for the prefix
  if (warp == 0) {
    const uint32_t sp = lane < kWalkWarps ? s_wsp[lane] : 0u;
    const uint32_t in = lane < kWalkWarps ? s_win[lane] : 0u;
    const uint32_t sp_incl = warp_inclusive_scan(sp), in_incl = warp_inclusive_scan(in);
    if (lane < kWalkWarps) {
      s_wsp[lane] = sp_incl - sp;
      s_win[lane] = in_incl - in;
    }
    const uint64_t tot_sp = __shfl_sync(0xffffffffu, sp_incl, 31), tot_in = __shfl_sync(0xffffffffu, in_incl, 31);
    volatile uint64_t* st = reinterpret_cast<volatile uint64_t*>(A.status);
    if (lane == 0) {
      st[tile] = (tile == 0 ? kWalkInclusive : kWalkAggregate) | walk_pack(tot_sp, tot_in);
      if (tot_in) atomicAdd(reinterpret_cast<unsigned long long*>(A.num_instances), (unsigned long long)tot_in);
    }
    uint64_t bsp = 0, bin = 0;
    int64_t j = tile - 1;
    int spins = 0;
    while (j >= 0) {  // uniform over the warp
      const int64_t idx = j - lane;
      const uint64_t v = idx >= 0 ? (uint64_t)st[idx] : (uint64_t)kWalkInclusive;  // before block 0: an inclusive zero
      const uint64_t flags = v & ~((1ull << 62) - 1);
      const unsigned incl_mask = __ballot_sync(0xffffffffu, flags == kWalkInclusive);
      const unsigned unready = __ballot_sync(0xffffffffu, flags == 0);
      const int first = incl_mask ? __ffs(incl_mask) - 1 : 32;  // nearest inclusive entry
      const unsigned need = first < 31 ? (2u << first) - 1u : 0xffffffffu;
      if (unready & need) {
        if (++spins > A.spin_limit) {
          if (lane == 0) atomicOr(A.err, A.pass_bit);
          break;
        }
        __nanosleep(64);
        continue;
      }
      uint64_t csp = ((need >> lane) & 1u) ? (v & kWalkField) : 0u;
      uint64_t cin = ((need >> lane) & 1u) ? ((v >> 31) & kWalkField) : 0u;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        csp += __shfl_xor_sync(0xffffffffu, csp, off);
        cin += __shfl_xor_sync(0xffffffffu, cin, off);
      }
      bsp += csp;
      bin += cin;
      if (first < 32) break;
      j -= 32;
    }
    if (lane == 0) {
      if (tile > 0) st[tile] = kWalkInclusive | walk_pack(bsp + tot_sp, bin + tot_in);
      s_before_sp = bsp;
      s_before_in = bin;
    }
  }
  __syncthreads();
  // 3. write the spans (cut at cap), with the row histogram
  if (live && wg * 32 < A.n) {  // uniform over the warp
    const uint64_t sbase = s_before_sp + s_wsp[warp], ibase = s_before_in + s_win[warp];
    const int64_t cap = A.cap;
    auto put = [&](uint64_t sidx, uint64_t ipos, int ty, int x0, int len, uint32_t gid) {
      if (ipos < (uint64_t)cap) {
        const int keep = (int)min((uint64_t)len, (uint64_t)cap - ipos);
        if (sidx < (uint64_t)cap) {  // (always, unless a look-back gave up)
          A.keys[sidx] = span_key(ty, x0, keep);
          A.vals[sidx] = gid;
          atomicAdd(&s_rows[ty], 1u);
        }
      } else {
        atomicMax(reinterpret_cast<unsigned long long*>(A.counters + 2), ~(unsigned long long)sidx);
      }
    };
    if (nsp <= (uint32_t)kWalkKeep) {
      for (uint32_t j = lane; j < nsp; j += 32) {
        const uint32_t k = s_key[warp][j];
        put(sbase + j, ibase + s_ioff[warp][j], (int)(k & 0xffu), span_x0(k), span_len(k), s_gid[warp][j]);
      }
    } else {  // walk again, writing as it goes
      uint64_t pos = ibase, spos = sbase;
      for (uint32_t rb = 0; rb < rows; rb += 32) {
        const uint32_t k = rb + lane;
        int o, ty, x0, x1;
        walk_row(w, row_incl, nr, k < rows ? k : rows - 1, &o, &ty, &x0, &x1);
        const uint32_t len = k < rows ? (uint32_t)(x1 - x0) : 0u;
        const uint32_t incl = warp_inclusive_scan(len);
        const unsigned has = __ballot_sync(0xffffffffu, len > 0u);
        if (len > 0u) put(spos + (uint64_t)__popc(has & lt), pos + (incl - len), ty, x0, (int)len, w.g[o]);
        pos += __shfl_sync(0xffffffffu, incl, 31);
        spos += (uint64_t)__popc(has);
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < A.tiles_y; i += kWalkThreads) {
    const uint32_t c = s_rows[i];
    if (c) atomicAdd(&A.hist[i], c);
  }
  // 4. the last block to finish sets the kept span count: all spans, or up to the first dropped
  __shared__ bool s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&A.counters[1], 1u) == (uint32_t)(blocks - 1);
  __syncthreads();
  if (s_last && threadIdx.x == 0) {
    __threadfence();
    const uint64_t last = *reinterpret_cast<volatile uint64_t*>(A.status + (blocks - 1));
    uint64_t total = last & kWalkField;
    const unsigned long long d = *reinterpret_cast<volatile unsigned long long*>(A.counters + 2);
    if (d != 0ull) total = min(total, (uint64_t)~d);
    *reinterpret_cast<int64_t*>(A.counters + 6) = (int64_t)total;
  }
}

// Words of the expansion's counter table: ceil(tiles_x / 2) lanes of packed 16-bit counters
// (column c: lane c mod L, half c / L), made odd so that the raking runs hit no bank twice, times
// the block's threads.
__host__ __device__ inline int span_lanes(int tiles_x) { return ((tiles_x + 1) / 2) | 1; }
// Spans per chunk: kSpanThreads times 4, 2 or 1, so that a chunk has fewer than 2^16 instances in
// either half of the table (at most spans x L).
__host__ __device__ inline int span_chunk(int tiles_x) {
  const int L = span_lanes(tiles_x);
  return kSpanThreads * (L * kSpanThreads * 4 < 65536 ? 4 : (L * kSpanThreads * 2 < 65536 ? 2 : 1));
}
inline size_t span_expand_smem(int tiles_x) {
  return sizeof(uint32_t) * ((size_t)span_lanes(tiles_x) * kSpanThreads + kSpanWindow + 2 * (kSpanMaxTiles + 1));
}

// One problem's span expansion.  A row's spans are cut into chunks of span_chunk(tiles_x) spans
// (the last one shorter); chunk b of the whole frame is chunk b - first(row) of its row, where
// first(row) counts the chunks of the rows before it.
struct SpanArgs {
  const uint32_t* keys;       // spans sorted by row
  const uint32_t* vals;
  const uint32_t* row_count;  // spans per row (the row sort's digit histogram)
  const int64_t* span_n;      // spans kept
  const uint32_t* err;
  int64_t* nptr;              // instance count: -1 when a sort gave up
  uint32_t* ctab;             // [chunks][tiles_x]: instances per column of each chunk
  uint32_t* row_total;        // [tiles_y] instances per row, then [tiles_y][tiles_x] per tile (zeroed first)
  uint2* ranges;
  uint32_t* point_list;
  uint32_t* tile_keys;        // optional
  int tiles_x, tiles_y;
  unsigned grid;
};

// Where chunk b lies: its row, its index in the row, its spans [s0, s1), and the instances of the
// rows before it (when row_total is given).  Returns false (for every thread) when b is past the
// frame's last chunk.  Synchronises the block; blockDim.x >= tiles_y.
struct ChunkPos {
  int row, index, chunks;  // chunks: the row's chunk count
  int64_t first, s0, s1;   // first: the frame index of the row's first chunk
  uint32_t row_base;
};

__device__ __forceinline__ bool locate_chunk(const uint32_t* __restrict__ row_count,
                                             const uint32_t* __restrict__ row_total, int tiles_y, int chunk,
                                             int64_t b, ChunkPos* pos) {
  __shared__ ChunkPos s_pos;
  __shared__ int s_found;
  if (threadIdx.x == 0) s_found = 0;
  const int r = threadIdx.x;
  const uint32_t cnt = r < tiles_y ? row_count[r] : 0u;
  const uint32_t nch = (cnt + (uint32_t)chunk - 1u) / (uint32_t)chunk;
  const uint32_t tot = (row_total != nullptr && r < tiles_y) ? row_total[r] : 0u;
  uint32_t all;
  const uint32_t ch_incl = block_inclusive_scan<uint32_t, kSpanThreads>(nch, &all);
  const uint32_t sp_incl = block_inclusive_scan<uint32_t, kSpanThreads>(cnt, &all);
  const uint32_t in_incl = block_inclusive_scan<uint32_t, kSpanThreads>(tot, &all);
  const int64_t first = (int64_t)(ch_incl - nch);
  if (r < tiles_y && b >= first && b < first + (int64_t)nch) {
    const int idx = (int)(b - first);
    const int64_t a = (int64_t)(sp_incl - cnt);
    s_pos.row = r;
    s_pos.index = idx;
    s_pos.chunks = (int)nch;
    s_pos.first = first;
    s_pos.s0 = a + (int64_t)idx * chunk;
    s_pos.s1 = min(a + (int64_t)cnt, s_pos.s0 + chunk);
    s_pos.row_base = in_incl - tot;
    s_found = 1;
  }
  __syncthreads();
  *pos = s_pos;
  return s_found != 0;
}

// Instances per column of each chunk (a difference array over the columns), summed into the
// row's and the tiles' totals.
// If a sort gave up waiting, the instance count becomes -1 and nothing else is written, so that no
// later kernel reads the lists and every reader of the count sees the failure.
__global__ void __launch_bounds__(kSpanThreads) span_count_kernel(const Batch<SpanArgs> b) {
  const SpanArgs& A = b.a[blockIdx.y];
  if (blockIdx.x >= A.grid) return;
  griddep_wait();
  const int tx = A.tiles_x;
  const int chunk = span_chunk(tx);
  if (*A.err != 0u) {  // a sort gave up: the instance count becomes -1 (the ranges stay empty)
    if (blockIdx.x == 0 && threadIdx.x == 0) *A.nptr = -1;
    return;
  }
  // chunks never exceed ceil(spans / chunk) + rows; the blocks stride over them
  const int64_t bound = (*A.span_n + chunk - 1) / chunk + A.tiles_y;
  uint32_t* tile_total = A.row_total + A.tiles_y;
  __shared__ int s_diff[kSpanMaxTiles + 1];
  for (int64_t b = blockIdx.x; b < bound; b += A.grid) {  // uniform over the block
    for (int c = threadIdx.x; c <= tx; c += kSpanThreads) s_diff[c] = 0;
    ChunkPos pos;
    if (!locate_chunk(A.row_count, nullptr, A.tiles_y, chunk, b, &pos)) return;
    for (int64_t i = pos.s0 + threadIdx.x; i < pos.s1; i += kSpanThreads) {
      const uint32_t k = A.keys[i];
      const int x0 = span_x0(k);
      atomicAdd(&s_diff[x0], 1);
      atomicAdd(&s_diff[min(x0 + span_len(k), tx)], -1);
    }
    __syncthreads();
    int tot;
    const int c = threadIdx.x;
    const int incl = block_inclusive_scan<int, kSpanThreads>(c < tx ? s_diff[c] : 0, &tot);
    if (c < tx) {
      A.ctab[(size_t)b * tx + c] = (uint32_t)incl;
      if (incl > 0) atomicAdd(&tile_total[pos.row * tx + c], (uint32_t)incl);
    }
    int all;
    block_inclusive_scan<int, kSpanThreads>(c < tx ? incl : 0, &all);
    if (c == 0 && all > 0) atomicAdd(&A.row_total[pos.row], (uint32_t)all);
  }
}

// Expands one chunk into its tiles' lists.  Thread t takes per = chunk / kSpanThreads consecutive
// spans and writes, in its own column of the counter table, how many of them cover each column (a
// difference array summed along the column).  An exclusive scan of the table in (column, thread)
// order then gives each (column, thread) its first position among the chunk's instances ordered by
// (column, depth); a span's instance at column c goes there plus the thread's earlier spans
// covering c.  The instances are staged in shared memory and each column's run is written
// contiguously at its place in the tile's list (a chunk with more than kSpanWindow instances
// writes them in place directly): after the instances of the
// rows before, of the row's tiles to the left, and of the row's earlier chunks at that column (all
// from the chunks' column counts).  The row's first chunk also writes the row's tile ranges.
__global__ void __launch_bounds__(kSpanThreads) span_expand_kernel(const Batch<SpanArgs> b) {
  const SpanArgs& A = b.a[blockIdx.y];
  if (blockIdx.x >= A.grid) return;
  griddep_wait();
  const int tx = A.tiles_x;
  const int chunk = span_chunk(tx), per = chunk / kSpanThreads;
  if (*A.err != 0u) return;
  // chunks never exceed ceil(spans / chunk) + rows; the blocks stride over them
  const int64_t bound = (*A.span_n + chunk - 1) / chunk + A.tiles_y;
  const uint32_t* tile_total = A.row_total + A.tiles_y;
  extern __shared__ __align__(16) uint32_t s_dyn[];
  const int L = span_lanes(tx);
  uint32_t* s_tab = s_dyn;                          // [L][kSpanThreads]
  uint32_t* s_stage = s_tab + L * kSpanThreads;     // [kSpanWindow]
  uint32_t* s_cpos = s_stage + kSpanWindow;         // [tx + 1] chunk position of each column's run
  uint32_t* s_goff = s_cpos + (kSpanMaxTiles + 1);  // [tx] list position of each column's run
  __shared__ uint32_t s_bp[kSpanThreads];
  const int t = threadIdx.x;
  for (int64_t bc = blockIdx.x; bc < bound; bc += A.grid) {  // uniform over the block
    ChunkPos pos;
    if (!locate_chunk(A.row_count, A.row_total, A.tiles_y, chunk, bc, &pos)) return;
    const int row = pos.row;
    const uint32_t tile0 = (uint32_t)row * (uint32_t)tx;
    {  // per column: the row's instances to the left of the tile, and the row's earlier chunks' at it
      const int g = kSpanThreads / tx;  // threads per column
      const int c = t % tx, k = t / tx;
      uint32_t before = 0;
      if (k < g)
        for (int j = k; j < pos.index; j += g) before += A.ctab[(size_t)(pos.first + j) * tx + c];
      s_bp[t] = before;
      __syncthreads();
      before = 0;
      const uint32_t all = t < tx ? tile_total[tile0 + t] : 0u;
      if (t < tx)
        for (int kk = 0; kk < g; ++kk) before += s_bp[kk * tx + t];
      uint32_t row_all;
      const uint32_t start = pos.row_base + block_inclusive_scan<uint32_t, kSpanThreads>(all, &row_all) - all;
      if (t < tx) {
        s_goff[t] = start + before;
        if (pos.index == 0) A.ranges[tile0 + t] = all > 0 ? make_uint2(start, start + all) : make_uint2(0u, 0u);
      }
    }
    int x0[kSpanPer], len[kSpanPer];
    uint32_t gid[kSpanPer];
    uint32_t carry = 0;  // my spans covering column L - 1 (the low half's last column)
#pragma unroll
    for (int i = 0; i < kSpanPer; ++i) {
      const int64_t s = pos.s0 + (int64_t)t * per + i;
      const bool in = i < per && s < pos.s1;
      const uint32_t k = in ? A.keys[s] : 0u;
      gid[i] = in ? A.vals[s] : 0u;
      x0[i] = span_x0(k);
      len[i] = in ? span_len(k) : 0;
      carry += (len[i] > 0 && x0[i] <= L - 1 && x0[i] + len[i] > L - 1) ? 1u : 0u;
    }
    // my column of the table: +1 where a span starts, -1 after it ends, then summed along the column
    for (int k = 0; k < L; ++k) s_tab[k * kSpanThreads + t] = 0u;
#pragma unroll
    for (int i = 0; i < kSpanPer; ++i) {
      if (len[i] == 0) continue;
      const int c0 = x0[i], c1 = x0[i] + len[i];
      const int h0 = c0 >= L;
      s_tab[(c0 - h0 * L) * kSpanThreads + t] += 1u << (16 * h0);
      if (c1 < 2 * L) {  // (columns tx .. 2L - 1 do not exist: they must count nothing)
        const int h1 = c1 >= L;
        s_tab[(c1 - h1 * L) * kSpanThreads + t] -= 1u << (16 * h1);
      }
    }
    {
      uint32_t run = carry << 16;  // the high half continues from column L - 1
      for (int k = 0; k < L; ++k) {
        run += s_tab[k * kSpanThreads + t];
        s_tab[k * kSpanThreads + t] = run;
      }
    }
    __syncthreads();
    uint32_t tot;
    {
      uint32_t* seg = s_tab + t * L;
      uint32_t sum = 0;
      for (int k = 0; k < L; ++k) sum += seg[k];
      uint32_t pre = block_inclusive_scan<uint32_t, kSpanThreads>(sum, &tot) - sum;
      for (int k = 0; k < L; ++k) {
        const uint32_t v = seg[k];
        seg[k] = pre;
        pre += v;
      }
    }
    __syncthreads();
    const uint32_t low = tot & 0xffffu, total = low + (tot >> 16);
    for (int c = t; c <= tx; c += kSpanThreads) {
      if (c == tx) {
        s_cpos[c] = total;
      } else {
        const int h = c >= L;
        s_cpos[c] = ((s_tab[(c - h * L) * kSpanThreads] >> (16 * h)) & 0xffffu) + (h ? low : 0u);
      }
    }
    __syncthreads();
    const int warp = t >> 5, lane = t & 31;
    uint32_t* __restrict__ out = A.point_list;
    uint32_t* __restrict__ out_keys = A.tile_keys;
    if (total <= (uint32_t)kSpanWindow) {  // uniform
      // Staged: each instance takes its (column, thread) entry, which then counts up for my next
      // span covering that column; then every column's run is copied out contiguously.
#pragma unroll
      for (int i = 0; i < kSpanPer; ++i)
        for (int c = x0[i]; c < x0[i] + len[i]; ++c) {
          const int h = c >= L;
          uint32_t* e = s_tab + (c - h * L) * kSpanThreads + t;
          const uint32_t w = *e;
          s_stage[((w >> (16 * h)) & 0xffffu) + (h ? low : 0u)] = gid[i];
          *e = w + (1u << (16 * h));
        }
      __syncthreads();
      for (int c = warp; c < tx; c += kSpanThreads / 32) {  // a warp per column run
        const uint32_t q0 = s_cpos[c], q1 = s_cpos[c + 1];
        const uint32_t g0 = s_goff[c];
        for (uint32_t q = q0 + lane; q < q1; q += 32) {
          out[g0 + (q - q0)] = s_stage[q];
          if (out_keys != nullptr) out_keys[g0 + (q - q0)] = tile0 + (uint32_t)c;
        }
      }
    } else {
      // A chunk of long spans, more instances than the stage holds: written in place directly.
#pragma unroll
      for (int i = 0; i < kSpanPer; ++i)
        for (int c = x0[i]; c < x0[i] + len[i]; ++c) {
          const int h = c >= L;
          uint32_t* e = s_tab + (c - h * L) * kSpanThreads + t;
          const uint32_t w = *e;
          const uint32_t q = ((w >> (16 * h)) & 0xffffu) + (h ? low : 0u);
          *e = w + (1u << (16 * h));
          const uint32_t g = s_goff[c] + (q - s_cpos[c]);
          out[g] = gid[i];
          if (out_keys != nullptr) out_keys[g] = tile0 + (uint32_t)c;
        }
    }
    __syncthreads();
  }
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

// ranges[t] = [first, end) of tile t in the sorted keys, (0, 0) for a tile without instances.  A
// block handles kRangeTiles consecutive tiles with one more warp than tiles: warp w finds where
// tile t0 + w starts, and tile t ends where tile t + 1 starts, so every warp does one search.  If a
// sort pass gave up waiting (*err), every range is empty and the instance count becomes -1, so
// that no later kernel reads the lists and every reader of the count sees the failure.
constexpr int kRangeTiles = 8;

struct RangesArgs {
  const uint32_t* keys;
  int64_t* nptr;
  int64_t cap;
  int num_tiles;
  const uint32_t* err;
  uint2* ranges;
  unsigned grid;
};

__global__ void __launch_bounds__((kRangeTiles + 1) * 32) ranges_kernel(const Batch<RangesArgs> b) {
  const RangesArgs& A = b.a[blockIdx.y];
  if (blockIdx.x >= A.grid) return;
  const uint32_t* __restrict__ keys = A.keys;
  int64_t* nptr = A.nptr;
  const int64_t cap = A.cap;
  const int num_tiles = A.num_tiles;
  const uint32_t* err = A.err;
  uint2* __restrict__ ranges = A.ranges;
  griddep_wait();
  __shared__ uint32_t s_start[kRangeTiles + 1];
  const int warp = threadIdx.x >> 5;
  const int t = blockIdx.x * kRangeTiles + warp;  // tile whose start this warp finds
  if (*err != 0u) {
    if (warp < kRangeTiles && t < num_tiles && (threadIdx.x & 31) == 0) ranges[t] = make_uint2(0u, 0u);
    if (blockIdx.x == 0 && threadIdx.x == 0) *nptr = -1;  // nothing else reads it after a failure
    return;
  }
  const int64_t n = element_count(nptr, 0, cap);
  if (t <= num_tiles) {  // whole warps
    const int64_t a = t < num_tiles ? warp_lower_bound(keys, n, (uint32_t)t) : n;
    if ((threadIdx.x & 31) == 0) s_start[warp] = (uint32_t)a;
  }
  __syncthreads();
  if (threadIdx.x < kRangeTiles) {
    const int tt = blockIdx.x * kRangeTiles + threadIdx.x;
    if (tt < num_tiles) {
      const uint32_t a = s_start[threadIdx.x], b = s_start[threadIdx.x + 1];
      ranges[tt] = b > a ? make_uint2(a, b) : make_uint2(0u, 0u);
    }
  }
}

__global__ void set_word_kernel(uint32_t* p, uint32_t v) { *p = v; }

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

// Test support: one 8-bit radix pass (the binning's look-back) whose tickets start at first_ticket,
// so that for first_ticket > 0 the blocks look back at tiles that no block will ever publish and
// each wait runs out after spin_limit rounds.  Workspace: an error word, then one sort's scratch.
size_t lookback_selftest_bytes(int64_t n) { return 256 + align256(sort_scratch_bytes(n, 8)); }

cudaError_t launch_lookback_selftest(const uint32_t* keys, const uint32_t* vals, uint32_t* keys_out,
                                     uint32_t* vals_out, int64_t n, uint32_t first_ticket, int spin_limit, char* ws,
                                     uint32_t** err_out, cudaStream_t st) {
  uint32_t* err = reinterpret_cast<uint32_t*>(ws);
  uint32_t* scratch = reinterpret_cast<uint32_t*>(ws + 256);
  *err_out = err;
  cudaError_t e = cudaMemsetAsync(ws, 0, lookback_selftest_bytes(n), st);
  if (e != cudaSuccess || n == 0) return e;
  // the pass's digit histogram, then its ticket counter moved past the first tiles
  uint32_t* kin[2] = {const_cast<uint32_t*>(keys), keys_out};
  uint32_t* vin[2] = {const_cast<uint32_t*>(vals), vals_out};
  const int64_t hist_blocks = std::min<int64_t>((n + kRadixThreads - 1) / kRadixThreads, 4 * device_sm_count());
  digit_hist_kernel<<<(unsigned)hist_blocks, kRadixThreads, 0, st>>>(keys, nullptr, n, n, 1, 8, scratch);
  set_word_kernel<<<1, 1, 0, st>>>(scratch + kMaxPasses * kBins, first_ticket);
  SortJob job{{kin[0], kin[1]}, {vin[0], vin[1]}, nullptr, n, n, 8, scratch, err, 0};
  int cur = 0;
  cudaError_t e2 = radix_sort(&job, 1, true, st, &cur, spin_limit);
  return e2 != cudaSuccess ? e2 : cudaGetLastError();
}

// The expansion's dynamic shared memory goes past the 48 KB default for wide images: opt in to
// the largest size it uses, once per device.
cudaError_t allow_span_expand_smem() {
  constexpr int kMaxDev = 64;
  static std::mutex mu;
  static bool done[kMaxDev] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDev) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  if (!done[dev]) {
    e = cudaFuncSetAttribute(span_expand_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)span_expand_smem(kSpanMaxTiles));
    if (e != cudaSuccess) return e;
    done[dev] = true;
  }
  return cudaSuccess;
}

// Words of the single-pass span walk's state: 64 counter words, then a 64-bit status per block.
size_t span_walk_words(int64_t n) { return 64 + 2 * (size_t)((n + kWalkThreads - 1) / kWalkThreads); }

BinPlan plan_bins(int64_t n, int64_t capacity, int width, int height) {
  BinPlan p;
  p.n = n;
  p.capacity = capacity;
  p.num_tiles = tiles_of(width) * tiles_of(height);
  int bits = 0;
  while ((int64_t(1) << bits) < p.num_tiles) ++bits;
  p.tile_bits = bits;
  const int tx = tiles_of(width), ty = tiles_of(height);
  p.spans = tx <= kSpanMaxTiles && ty <= kSpanMaxTiles;
  p.row_bits = 0;
  while ((1 << p.row_bits) < ty) ++p.row_bits;
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
  p.off_sort_t = off; off += align256(sort_scratch_bytes(capacity, p.spans ? p.row_bits : bits));
  p.off_partials = off; off += align256(sizeof(uint64_t) * p.partial_cap);
  p.off_svals = p.off_walk = p.off_ctab = p.off_rowtot = 0;
  if (p.spans) {
    p.off_svals = off; off += align256(sizeof(uint32_t) * capacity);
    p.off_walk = off; off += align256(sizeof(uint32_t) * span_walk_words(n));
    const int64_t chunks = (capacity + span_chunk(tx) - 1) / span_chunk(tx) + ty;  // at most
    p.off_ctab = off; off += align256(sizeof(uint32_t) * (size_t)chunks * tx);
    p.off_rowtot = off; off += align256(sizeof(uint32_t) * (size_t)ty * (1 + tx));
  }
  p.total = off;
  return p;
}

cudaError_t launch_bin_sort_batch(const BinRequest* reqs, int count, cudaStream_t st) {
  if (count < 1 || count > kMaxBatch) return cudaErrorInvalidValue;
  // Workspace carve-up of every request.
  struct Work {
    int64_t n;
    int tiles_x, tiles_y;
    uint32_t *dkeys[2], *dvals[2], *sort_d, *sort_t, *err, *out_keys, *ikeys[2], *ivals[2];
    uint64_t *first, *partials;
    uint32_t *skeys[2], *svals[2], *ctab, *rowtot, *walk;  // span binning
    int64_t* span_n;
    const ushort4* rect;
    const float2* m2;
    const float4* co;
    const uint32_t* order;
  } W[kMaxBatch];
  cudaError_t e = cudaSuccess;
  BatchLaunch<ClearJob> clears;
  for (int j = 0; j < count; ++j) {
    const BinRequest& R = reqs[j];
    const BinPlan& plan = R.plan;
    char* ws = R.ws;
    Work& w = W[j];
    w.n = plan.n;
    w.tiles_x = tiles_of(R.view.width);
    w.tiles_y = tiles_of(R.view.height);
    for (int k = 0; k < 2; ++k) {
      w.dkeys[k] = reinterpret_cast<uint32_t*>(ws + plan.off_dkeys[k]);
      w.dvals[k] = reinterpret_cast<uint32_t*>(ws + plan.off_dvals[k]);
    }
    w.first = reinterpret_cast<uint64_t*>(ws + plan.off_first);
    w.sort_d = reinterpret_cast<uint32_t*>(ws + plan.off_sort_d);
    w.sort_t = reinterpret_cast<uint32_t*>(ws + plan.off_sort_t);
    w.err = reinterpret_cast<uint32_t*>(ws + plan.off_err);
    w.partials = reinterpret_cast<uint64_t*>(ws + plan.off_partials);
    w.rect = reinterpret_cast<const ushort4*>(R.proj.rect);
    w.m2 = reinterpret_cast<const float2*>(R.proj.mean2d);
    w.co = reinterpret_cast<const float4*>(R.proj.conic_opacity);
    // the instance buffers, ordered so that the tile passes end in the outputs
    const int passes = radix_pass_count(plan.tile_bits);
    w.out_keys = R.out.tile_keys ? R.out.tile_keys : reinterpret_cast<uint32_t*>(ws + plan.off_ikeys[1]);
    uint32_t* wk0 = reinterpret_cast<uint32_t*>(ws + plan.off_ikeys[0]);
    uint32_t* wv0 = reinterpret_cast<uint32_t*>(ws + plan.off_ivals);
    const bool even = passes % 2 == 0;
    w.ikeys[0] = even ? w.out_keys : wk0;
    w.ivals[0] = even ? R.out.point_list : wv0;
    w.ikeys[1] = even ? wk0 : w.out_keys;
    w.ivals[1] = even ? wv0 : R.out.point_list;
    if (plan.spans) {  // spans ping-pong in the workspace; the expansion writes the outputs
      w.skeys[0] = wk0;
      w.skeys[1] = reinterpret_cast<uint32_t*>(ws + plan.off_ikeys[1]);
      w.svals[0] = wv0;
      w.svals[1] = reinterpret_cast<uint32_t*>(ws + plan.off_svals);
      w.walk = reinterpret_cast<uint32_t*>(ws + plan.off_walk);
      w.span_n = reinterpret_cast<int64_t*>(w.walk + 6);
      w.ctab = reinterpret_cast<uint32_t*>(ws + plan.off_ctab);
      w.rowtot = reinterpret_cast<uint32_t*>(ws + plan.off_rowtot);
    }
    ClearJob c;
    // (with Gaussians, the ranges or span starts kernel writes every tile's range)
    c.ptr[0] = (w.n == 0 || plan.spans) ? R.out.ranges : nullptr; c.words[0] = 2 * (size_t)plan.num_tiles;
    c.ptr[1] = w.err; c.words[1] = 1;
    c.ptr[2] = w.n == 0 ? reinterpret_cast<uint32_t*>(R.out.num_instances) : (plan.spans ? w.rowtot : nullptr);
    c.words[2] = w.n == 0 ? 2 : (size_t)w.tiles_y * (1 + w.tiles_x);
    c.ptr[3] = w.n > 0 ? w.sort_d : nullptr; c.words[3] = sort_scratch_bytes(w.n, 32) / 4;
    c.ptr[4] = w.n > 0 ? w.sort_t : nullptr;
    c.words[4] = sort_scratch_bytes(plan.capacity, plan.spans ? plan.row_bits : plan.tile_bits) / 4;
    // span binning: the walk's counters and status words, and K (which the walk adds up)
    c.ptr[5] = (w.n > 0 && plan.spans) ? w.walk : nullptr; c.words[5] = span_walk_words(w.n);
    c.ptr[6] = (w.n > 0 && plan.spans) ? reinterpret_cast<uint32_t*>(R.out.num_instances) : nullptr; c.words[6] = 2;
    size_t most = 0;
    for (int k = 0; k < ClearJob::kSlots; ++k) most = std::max(most, c.ptr[k] ? c.words[k] : 0);
    c.grid = (unsigned)std::max<size_t>(1, std::min<size_t>((most + 255) / 256, 4 * (size_t)device_sm_count()));
    clears.add(c);
  }
  e = launch_batch(clear_kernel, clears, 256, 0, st);
  for (int j = 0; j < count && e == cudaSuccess; ++j) {  // test support
    if (reqs[j].inject_err != 0u) {  // as if a pass had given up waiting
      set_word_kernel<<<1, 1, 0, st>>>(W[j].err, reqs[j].inject_err);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess && reqs[j].walk_ticket != 0u && reqs[j].plan.spans && W[j].n > 0) {
      set_word_kernel<<<1, 1, 0, st>>>(W[j].walk, reqs[j].walk_ticket);  // the span walk's first ticket
      e = cudaGetLastError();
    }
  }
  if (e != cudaSuccess) return e;
  // Only the requests with Gaussians go on (the others are complete: no instances, empty ranges).
  int live[kMaxBatch], nl = 0;
  for (int j = 0; j < count; ++j)
    if (W[j].n > 0) live[nl++] = j;
  if (nl == 0) return cudaSuccess;
  // 1. Gaussians by float32 depth (stable; culled ones last).
  BatchLaunch<DepthKeysArgs> keys;
  SortJob dsort[kMaxBatch];
  int dcur[kMaxBatch];
  for (int i = 0; i < nl; ++i) {
    Work& w = W[live[i]];
    DepthKeysArgs a{reqs[live[i]].proj.depth, w.rect, w.n, w.dkeys[0], w.dvals[0], w.sort_d,
                    reqs[live[i]].plan.spans ? w.walk + 4 : nullptr,
                    (unsigned)std::min<int64_t>((w.n + 4 * kRadixThreads - 1) / (4 * kRadixThreads),
                                                2 * device_sm_count())};
    keys.add(a);
    dsort[i] = SortJob{{w.dkeys[0], w.dkeys[1]}, {w.dvals[0], w.dvals[1]}, nullptr, w.n, w.n, 32, w.sort_d, w.err, 0};
  }
  if ((e = launch_batch(depth_keys_kernel, keys, kRadixThreads, 0, st)) != cudaSuccess) return e;
  if ((e = radix_sort(dsort, nl, true, st, dcur)) != cudaSuccess) return e;
  // 2. Instance path: kept tiles per warp of 32 depth-ordered Gaussians (row spans); first
  //    instance of each warp and K; the instances in depth order, with the tile-digit histograms.
  //    Span binning: the single-pass span walk (spans in depth order, K, the row histogram).
  BatchLaunch<WalkArgs> walks;
  BatchLaunch<SpanWalkArgs> swalks;
  ScanArgs<uint32_t, uint64_t> scans[kMaxBatch];
  int nscan = 0;
  for (int i = 0; i < nl; ++i) {
    Work& w = W[live[i]];
    const BinRequest& R = reqs[live[i]];
    w.order = w.dvals[dcur[i]];
    if (R.plan.spans) {
      SpanWalkArgs a{};
      a.order = w.order; a.rect = w.rect; a.mean2d = w.m2; a.conic_opacity = w.co; a.n = w.n;
      a.tiles_x = w.tiles_x; a.tiles_y = w.tiles_y; a.err = w.err;
      a.pass_bit = 1u << kMaxPasses; a.spin_limit = R.spin_limit > 0 ? R.spin_limit : kLookbackSpins;
      a.cap = R.plan.capacity;
      a.keys = w.skeys[0]; a.vals = w.svals[0];
      a.hist = w.sort_t;
      a.num_instances = R.out.num_instances;
      a.counters = w.walk;
      a.status = reinterpret_cast<uint64_t*>(w.walk + 64);
      a.grid = (unsigned)((w.n + kWalkThreads - 1) / kWalkThreads);
      swalks.add(a);
      continue;
    }
    const int64_t nwarps = (w.n + 31) / 32;
    WalkArgs a{};
    a.order = w.order; a.rect = w.rect; a.mean2d = w.m2; a.conic_opacity = w.co; a.n = w.n;
    a.tiles_x = w.tiles_x; a.tiles_y = w.tiles_y; a.err = w.err;
    a.wcount = w.dkeys[dcur[i] ^ 1];
    a.wfirst = w.first; a.cap = R.plan.capacity;
    a.hist = w.sort_t;
    a.keys = w.ikeys[0]; a.vals = w.ivals[0];
    a.passes = radix_pass_count(R.plan.tile_bits); a.width = radix_digit_width(R.plan.tile_bits);
    a.grid = (unsigned)((nwarps + kWalkWarps - 1) / kWalkWarps);
    walks.add(a);
    scans[nscan++] = ScanArgs<uint32_t, uint64_t>{a.wcount, nwarps, w.first, reinterpret_cast<uint64_t*>(w.partials),
                                                  R.out.num_instances, 0};
  }
  if ((e = launch_batch(span_walk_kernel, swalks, kWalkThreads, 0, st)) != cudaSuccess) return e;
  if ((e = launch_batch(walk_count_kernel, walks, kWalkThreads, 0, st)) != cudaSuccess) return e;
  if ((e = exclusive_scan(scans, nscan, st)) != cudaSuccess) return e;
  if ((e = launch_batch(walk_emit_kernel, walks, kWalkThreads, 0, st)) != cudaSuccess) return e;
  // 3. Stable sort by tile id (instance path) or by row (span binning).
  SortJob tsort[kMaxBatch];
  int tcur[kMaxBatch];
  for (int i = 0; i < nl; ++i) {
    Work& w = W[live[i]];
    const BinRequest& R = reqs[live[i]];
    if (R.plan.spans)  // (bit kMaxPasses of the error word is the span walk's)
      tsort[i] = SortJob{{w.skeys[0], w.skeys[1]}, {w.svals[0], w.svals[1]}, w.span_n, 0,
                         R.plan.capacity, R.plan.row_bits, w.sort_t, w.err, kMaxPasses + 1};
    else
      tsort[i] = SortJob{{w.ikeys[0], w.ikeys[1]}, {w.ivals[0], w.ivals[1]}, R.out.num_instances, 0,
                         R.plan.capacity, R.plan.tile_bits, w.sort_t, w.err, kMaxPasses};
  }
  if ((e = radix_sort(tsort, nl, true, st, tcur)) != cudaSuccess) return e;
  // 4. Tile ranges (instance records), or the span expansion into the tile lists.
  BatchLaunch<RangesArgs> ranges;
  BatchLaunch<SpanArgs> scnt, sexp;
  size_t sexp_smem = 0;
  for (int i = 0; i < nl; ++i) {
    Work& w = W[live[i]];
    const BinRequest& R = reqs[live[i]];
    if (R.plan.spans) {
      const int64_t chunks = (R.plan.capacity + span_chunk(w.tiles_x) - 1) / span_chunk(w.tiles_x) + w.tiles_y;
      SpanArgs a{w.skeys[tcur[i]], w.svals[tcur[i]], w.sort_t, w.span_n, w.err, R.out.num_instances, w.ctab,
                 w.rowtot, reinterpret_cast<uint2*>(R.out.ranges), R.out.point_list, R.out.tile_keys,
                 w.tiles_x, w.tiles_y, (unsigned)chunks};
      a.grid = (unsigned)std::min<int64_t>(chunks, 8 * (int64_t)device_sm_count());
      scnt.add(a);
      a.grid = (unsigned)std::min<int64_t>(chunks, 3 * (int64_t)device_sm_count());
      sexp.add(a);
      sexp_smem = std::max(sexp_smem, span_expand_smem(w.tiles_x));
    } else {
      const int64_t blocks = (R.plan.num_tiles + kRangeTiles - 1) / kRangeTiles;
      RangesArgs a{w.out_keys, R.out.num_instances, R.plan.capacity, (int)R.plan.num_tiles, w.err,
                   reinterpret_cast<uint2*>(R.out.ranges), (unsigned)blocks};
      ranges.add(a);
    }
  }
  if ((e = launch_batch(ranges_kernel, ranges, (kRangeTiles + 1) * 32, 0, st)) != cudaSuccess) return e;
  if (sexp.count > 0) {
    if ((e = allow_span_expand_smem()) != cudaSuccess) return e;
    if ((e = launch_batch(span_count_kernel, scnt, kSpanThreads, 0, st)) != cudaSuccess) return e;
    if ((e = launch_batch(span_expand_kernel, sexp, kSpanThreads, sexp_smem, st)) != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

cudaError_t launch_bin_sort(const sdgs_projected& proj, const sdgs_view& v, const BinPlan& plan, char* ws,
                            const sdgs_bins& out, cudaStream_t st, uint32_t inject_err, uint32_t walk_ticket,
                            int spin_limit) {
  const BinRequest r{proj, v, plan, ws, out, inject_err, walk_ticket, spin_limit};
  return launch_bin_sort_batch(&r, 1, st);
}

}  // namespace sdgs
