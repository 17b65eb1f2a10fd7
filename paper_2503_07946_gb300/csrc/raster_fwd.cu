// Forward tile rasteriser (Sec. 4.4; the 3DGS blending rules).
//
// One 128-thread block per 16x16 tile; each thread owns two pixels of one column, rows r and
// r + 8, so every Gaussian fetched from shared memory is evaluated twice.  The tile's sorted
// instances (only Gaussians that may reach the tile, see tile_reach.cuh) are staged 128 at a time
// in shared memory; each pixel walks them front to back.  The block leaves once every pixel has
// stopped.
#include "raster_common.cuh"

namespace sdgs {

namespace {

constexpr int kThreads = kTilePixels / 2;

struct FwdArgs {
  const float2* mean2d;
  const float4* conic_opacity;
  const float* rgb;
  const uint32_t* point_list;
  const uint2* ranges;
  int width, height, tiles_x;
  float bg[3];
  float* image;
  float* final_T;
  uint32_t* n_contrib;
  unsigned long long* n_evaluated;  // optional work counter
};

struct Pixel {
  float T = 1.f, c0 = 0.f, c1 = 0.f, c2 = 0.f;
  uint32_t last = 0, evaluated = 0;
  bool done;
};

// One (pixel, Gaussian) evaluation written without branches, so that a thread's two pixels
// interleave: the pixel takes the Gaussian iff it is still running, the exponent is <= 0 and
// alpha >= 1/255; if that would take T below 1e-4 the pixel stops instead (without blending).
template <bool kCount>
__device__ __forceinline__ void blend(Pixel& px, const float4& q, const float4& c, float dx, float dy,
                                      uint32_t pos1) {
  const float p2 = splat_power2(q, dx, dy);
  const float al = fminf(kAlphaMax, __fmul_rn(q.w, ex2_approx(p2)));
  const float Tn = __fmul_rn(px.T, __fsub_rn(1.f, al));
  const bool live = !px.done;
  const bool hit = live && p2 <= 0.f && al >= kAlphaMin;
  const bool stop = hit && Tn < kTMin;
  const bool take = hit && !stop;
  const float w = take ? al * px.T : 0.f;
  if (kCount) px.evaluated += live ? 1u : 0u;
  px.c0 += c.x * w;
  px.c1 += c.y * w;
  px.c2 += c.z * w;
  px.T = take ? Tn : px.T;
  px.last = take ? pos1 : px.last;
  px.done = px.done || stop;
}

template <bool kCount>
__global__ void __launch_bounds__(kThreads) render_fwd_kernel(const FwdArgs a) {
  __shared__ float2 s_xy[kThreads];
  __shared__ float4 s_q[kThreads];
  __shared__ float4 s_rgb[kThreads];

  const int tile = blockIdx.x;
  const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
  const int lane = threadIdx.x & 31;
  const int px = tx * kTile + (threadIdx.x & (kTile - 1));
  const int py0 = ty * kTile + (threadIdx.x / kTile);
  const int py1 = py0 + kTile / 2;
  const float fx = (float)px + 0.5f, fy0 = (float)py0 + 0.5f, fy1 = (float)py1 + 0.5f;
  const uint2 range = a.ranges[tile];
  const int n = (int)(range.y - range.x);

  Pixel p0, p1;
  p0.done = !(px < a.width && py0 < a.height);
  p1.done = !(px < a.width && py1 < a.height);
  for (int base = 0; base < n; base += kThreads) {
    if (__syncthreads_count(p0.done && p1.done) == kThreads) break;
    // stage the next 128 instances of the tile's list
    const int j = base + threadIdx.x;
    if (j < n) {
      const uint32_t g = a.point_list[range.x + j];
      s_xy[threadIdx.x] = a.mean2d[g];
      s_q[threadIdx.x] = scaled_conic(a.conic_opacity[g]);
      s_rgb[threadIdx.x] = make_float4(a.rgb[3 * g + 0], a.rgb[3 * g + 1], a.rgb[3 * g + 2], 0.f);
    }
    const int cnt = min(kThreads, n - base);
    __syncthreads();
    if (!(p0.done && p1.done)) {
      // Entries past cnt are never read: the batch is padded by predication.  The stop test runs
      // every 4 Gaussians; a stopped pixel ignores the rest (blend is a no-op once done).
      for (int k0 = 0; k0 < cnt; k0 += 4) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int k = k0 + u;
          if (k < cnt) {
            const float2 m = s_xy[k];
            const float4 q = s_q[k];
            const float4 c = s_rgb[k];
            const uint32_t pos1 = (uint32_t)(base + k) + 1u;
            // offsets exactly as the backward forms them, so both passes take the same decisions
            const float dx = fx - m.x;
            blend<kCount>(p0, q, c, dx, fy0 - m.y, pos1);
            blend<kCount>(p1, q, c, dx, fy1 - m.y, pos1);
          }
        }
        if (p0.done && p1.done) break;
      }
    }
  }
  if (kCount) {
    unsigned long long e = (unsigned long long)p0.evaluated + p1.evaluated;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
    if (lane == 0 && e) atomicAdd(a.n_evaluated, e);
  }
  const Pixel* pp[2] = {&p0, &p1};
  const int rows[2] = {py0, py1};
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    if (px < a.width && rows[r] < a.height) {
      const int pix = rows[r] * a.width + px;
      const Pixel& q = *pp[r];
      a.image[3 * pix + 0] = q.c0 + q.T * a.bg[0];
      a.image[3 * pix + 1] = q.c1 + q.T * a.bg[1];
      a.image[3 * pix + 2] = q.c2 + q.T * a.bg[2];
      a.final_T[pix] = q.T;
      a.n_contrib[pix] = q.last;
    }
  }
}

}  // namespace

cudaError_t launch_render_fwd(const sdgs_projected& p, const sdgs_bins& b, const sdgs_view& v,
                              float* image, float* final_T, uint32_t* n_contrib,
                              uint64_t* n_evaluated, cudaStream_t st) {
  FwdArgs a;
  a.mean2d = reinterpret_cast<const float2*>(p.mean2d);
  a.conic_opacity = reinterpret_cast<const float4*>(p.conic_opacity);
  a.rgb = p.rgb;
  a.point_list = b.point_list;
  a.ranges = reinterpret_cast<const uint2*>(b.ranges);
  a.width = v.width;
  a.height = v.height;
  a.tiles_x = tiles_of(v.width);
  for (int c = 0; c < 3; ++c) a.bg[c] = v.bg[c];
  a.image = image;
  a.final_T = final_T;
  a.n_contrib = n_contrib;
  a.n_evaluated = reinterpret_cast<unsigned long long*>(n_evaluated);
  const int tiles = a.tiles_x * tiles_of(v.height);
  if (tiles == 0) return cudaSuccess;
  if (n_evaluated != nullptr)
    render_fwd_kernel<true><<<tiles, kThreads, 0, st>>>(a);
  else
    render_fwd_kernel<false><<<tiles, kThreads, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace sdgs
