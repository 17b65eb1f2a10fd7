// Forward tile rasteriser: one 256-thread block per 16x16 tile, one pixel per thread.
// The tile's sorted instances are staged through shared memory in batches of 256; every pixel
// walks the batch front to back (Sec. 4.3 depth-aware opacity blending with the 3DGS rules).
// The block leaves as soon as every pixel of the tile has stopped.
#include "common.cuh"

namespace sdgs {

namespace {

constexpr int kThreads = kTilePixels;
constexpr float kLog2e = 1.4426950408889634f;

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

__global__ void __launch_bounds__(kThreads) render_fwd_kernel(const FwdArgs a) {
  __shared__ float2 s_xy[kThreads];
  __shared__ float4 s_q[kThreads];  // (-a/2, -b, -c/2) * log2(e), alpha_cond
  __shared__ float s_rgb[3][kThreads];

  const int tile = blockIdx.x;
  const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
  const int px = tx * kTile + (threadIdx.x & (kTile - 1));
  const int py = ty * kTile + (threadIdx.x / kTile);
  const bool inside = px < a.width && py < a.height;
  const float fx = (float)px + 0.5f, fy = (float)py + 0.5f;
  const uint2 range = a.ranges[tile];
  const int n = (int)(range.y - range.x);

  bool done = !inside;
  float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
  uint32_t last = 0;
  uint32_t evaluated = 0;
  for (int base = 0; base < n; base += kThreads) {
    if (__syncthreads_count(done) == kThreads) break;
    const int j = base + threadIdx.x;
    if (j < n) {
      const uint32_t g = a.point_list[range.x + j];
      s_xy[threadIdx.x] = a.mean2d[g];
      const float4 q = a.conic_opacity[g];
      s_q[threadIdx.x] = make_float4(-0.5f * kLog2e * q.x, -kLog2e * q.y, -0.5f * kLog2e * q.z, q.w);
      s_rgb[0][threadIdx.x] = a.rgb[3 * g + 0];
      s_rgb[1][threadIdx.x] = a.rgb[3 * g + 1];
      s_rgb[2][threadIdx.x] = a.rgb[3 * g + 2];
    }
    __syncthreads();
    if (!done) {
      const int cnt = min(kThreads, n - base);
      int k = 0;
      for (; k < cnt; ++k) {
        const float2 xy = s_xy[k];
        const float4 q = s_q[k];
        const float dx = fx - xy.x, dy = fy - xy.y;
        const float p2 = q.x * dx * dx + q.z * dy * dy + q.y * dx * dy;
        if (p2 > 0.f) continue;
        const float al = fminf(kAlphaMax, q.w * exp2f(p2));
        if (al < kAlphaMin) continue;
        const float Tn = T * (1.f - al);
        if (Tn < kTMin) {
          done = true;
          ++k;  // the stopping Gaussian was evaluated too
          break;
        }
        const float w = al * T;
        C0 += s_rgb[0][k] * w;
        C1 += s_rgb[1][k] * w;
        C2 += s_rgb[2][k] * w;
        T = Tn;
        last = (uint32_t)(base + k + 1);
      }
      evaluated += (uint32_t)k;
    }
  }
  if (a.n_evaluated != nullptr) {
    unsigned long long e = evaluated;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
    if ((threadIdx.x & 31) == 0 && e) atomicAdd(a.n_evaluated, e);
  }
  if (inside) {
    const int pix = py * a.width + px;
    a.image[3 * pix + 0] = C0 + T * a.bg[0];
    a.image[3 * pix + 1] = C1 + T * a.bg[1];
    a.image[3 * pix + 2] = C2 + T * a.bg[2];
    a.final_T[pix] = T;
    a.n_contrib[pix] = last;
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
  render_fwd_kernel<<<tiles, kThreads, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace sdgs
