// Forward tile rasteriser (Sec. 4.4; the 3DGS blending rules).
//
// One 128-thread block per 16x16 tile; each thread owns two pixels of one column, rows r and
// r + 8, so every Gaussian fetched from shared memory is evaluated twice.  The tile's sorted
// instances (only Gaussians that may reach the tile, see tile_reach.cuh) are staged 128 at a time
// in shared memory; each pixel walks them front to back.  The block leaves once every pixel has
// stopped.  A batch in which no staged Gaussian can reach the 0.99 clamp of alpha at any pixel of
// the tile (clamp_free) is blended without the clamp.
#include <type_traits>

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
  uint32_t n;  // Gaussians in the records; a list entry >= n (never written by binning) is skipped
  float bg[3];
  float* image;
  float* final_T;
  uint32_t* n_contrib;
  unsigned long long* n_evaluated;  // optional work counters: [0] evaluations, [1] contributions
};

// The two pixels of a thread (rows r and r + 8 of one column) as pairs, so that the arithmetic
// they share runs as paired FP32 operations (each element correctly rounded, identical to the
// scalar operations the backward uses).
struct PixelPair {
  float2 T = make_float2(1.f, 1.f), c0 = make_float2(0.f, 0.f), c1 = make_float2(0.f, 0.f),
         c2 = make_float2(0.f, 0.f);
  uint32_t last0 = 0, last1 = 0, evaluated = 0, contributed = 0;
  bool done0, done1;
};

// One Gaussian evaluated at both pixels, without branches: a pixel takes the Gaussian iff it is
// still running and alpha >= 1/255; if that would take T below 1e-4 the pixel stops instead
// (without blending).  The exponent is qa dx^2 + dy (qc dy + qb dx), as in splat_power2; staged
// conics are positive definite (others get opacity 0), so it is <= 0 but for FP32 rounding at a
// pixel on the centre, where alpha is then alpha_cond (the FP64 oracle takes the Gaussian there).
// kClamp = false: the caller knows that alpha_cond * exp2(exponent) <= 0.99 for this Gaussian at
// both pixels (see clamp_free), so the 0.99 clamp would return its argument and is left out.
template <bool kCount, bool kClamp = true>
__device__ __forceinline__ void blend2(PixelPair& px, const float4& q, const float4& c, float dx, float2 dy,
                                       uint32_t pos1) {
  const float a = __fmul_rn(__fmul_rn(q.x, dx), dx);
  const float bx = __fmul_rn(q.y, dx);
  const float2 t = __ffma2_rn(make_float2(q.z, q.z), dy, make_float2(bx, bx));
  const float2 p2 = __ffma2_rn(dy, t, make_float2(a, a));
  const float2 e = make_float2(ex2_approx(p2.x), ex2_approx(p2.y));
  const float2 m = __fmul2_rn(make_float2(q.w, q.w), e);
  const float2 al = kClamp ? make_float2(fminf(kAlphaMax, m.x), fminf(kAlphaMax, m.y)) : m;
  const float2 aT = __fmul2_rn(al, px.T);
  const float2 Tn = __fadd2_rn(px.T, make_float2(-aT.x, -aT.y));  // T (1 - alpha) as T - alpha T
  const bool hit0 = !px.done0 && al.x >= kAlphaMin;
  const bool hit1 = !px.done1 && al.y >= kAlphaMin;
  const bool stop0 = hit0 && Tn.x < kTMin, stop1 = hit1 && Tn.y < kTMin;
  const bool take0 = hit0 && !stop0, take1 = hit1 && !stop1;
  if (kCount) {
    px.evaluated += (px.done0 ? 0u : 1u) + (px.done1 ? 0u : 1u);
    px.contributed += (take0 ? 1u : 0u) + (take1 ? 1u : 0u);
  }
  const float2 w = make_float2(take0 ? aT.x : 0.f, take1 ? aT.y : 0.f);
  px.c0 = __ffma2_rn(make_float2(c.x, c.x), w, px.c0);
  px.c1 = __ffma2_rn(make_float2(c.y, c.y), w, px.c1);
  px.c2 = __ffma2_rn(make_float2(c.z, c.z), w, px.c2);
  px.T = __fadd2_rn(px.T, make_float2(-w.x, -w.y));  // Tn where taken, T - 0 = T elsewhere
  px.last0 = take0 ? pos1 : px.last0;
  px.last1 = take1 ? pos1 : px.last1;
  px.done0 = px.done0 || stop0;
  px.done1 = px.done1 || stop1;
}

// Whether the 0.99 clamp of alpha cannot act for staged Gaussian (m, q) at any pixel centre of the
// tile whose first pixel centre is (x0, y0).  The exponent is evaluated as in blend2 from the
// rounded offsets dx, dy; for a positive-definite conic its exact value at those offsets is <= 0,
// and the three roundings of a, bx, t and the final sum add at most
// gamma_3 * S, S = |qa| Dx^2 + |qb| Dx Dy + |qc| Dy^2 with Dx, Dy bounds of |dx|, |dy| over the
// tile (gamma_3 = 3u / (1 - 3u), u = 2^-24).  With S <= 6e4 that is below 0.0108, so exp2 of the
// computed exponent is below 2^0.0108 = 1.0075, ex2.approx adds a relative error far below 1e-6,
// and alpha_cond <= 0.98 keeps alpha_cond * exp2 <= 0.9874 < 0.99.  (S is formed in FP32 from
// values that bound the true ones; NaN or infinite inputs fail the test.)
__device__ __forceinline__ bool clamp_free(float2 m, float4 q, float x0, float y0) {
  const float Dx = fmaxf(fabsf(x0 - m.x), fabsf(x0 + 15.f - m.x)) * 1.0001f;
  const float Dy = fmaxf(fabsf(y0 - m.y), fabsf(y0 + 15.f - m.y)) * 1.0001f;
  const float S = (fabsf(q.x) * Dx * Dx + fabsf(q.y) * Dx * Dy + fabsf(q.z) * Dy * Dy) * 1.0001f;
  return q.w <= 0.98f && S <= 6e4f;
}

template <bool kCount>
__global__ void __launch_bounds__(kThreads) render_fwd_kernel(const FwdArgs a) {
  griddep_wait();
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

  PixelPair pp;
  pp.done0 = !(px < a.width && py0 < a.height);
  pp.done1 = !(px < a.width && py1 < a.height);
  const float2 fy = make_float2(fy0, fy1);
  for (int base = 0; base < n; base += kThreads) {
    if (__syncthreads_count(pp.done0 && pp.done1) == kThreads) break;
    // stage the next 128 instances of the tile's list
    const int j = base + threadIdx.x;
    bool no_clamp = true;  // the 0.99 clamp cannot act for this thread's staged Gaussian
    if (j < n) {
      const uint32_t g = a.point_list[range.x + j];
      if (g < a.n) {
        const float2 m = a.mean2d[g];
        const float4 q = scaled_conic(pd_or_transparent(a.conic_opacity[g]));
        s_xy[threadIdx.x] = m;
        s_q[threadIdx.x] = q;
        s_rgb[threadIdx.x] = make_float4(a.rgb[3 * g + 0], a.rgb[3 * g + 1], a.rgb[3 * g + 2], 0.f);
        no_clamp = clamp_free(m, q, (float)(tx * kTile) + 0.5f, (float)(ty * kTile) + 0.5f);
      } else {  // opacity 0: every pixel skips it
        s_xy[threadIdx.x] = make_float2(0.f, 0.f);
        s_q[threadIdx.x] = make_float4(0.f, 0.f, 0.f, 0.f);
        s_rgb[threadIdx.x] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    const int cnt = min(kThreads, n - base);
    // whether the whole batch can run without the clamp (uniform over the block)
    const bool batch_no_clamp = __syncthreads_and(no_clamp) != 0;
    if (!(pp.done0 && pp.done1)) {
      // A full batch runs as straight-line groups of 8 Gaussians with the stop test after each
      // group; the tile's last, partial batch in groups of 4 with bound checks (entries past cnt
      // are never read).  A stopped pixel ignores the rest (blend2 is a no-op for it).
      auto run = [&](auto clamp) {
        constexpr bool kClamp = decltype(clamp)::value;
        auto one = [&](int k) {
          const float2 m = s_xy[k];
          const float4 q = s_q[k];
          const float4 c = s_rgb[k];
          const uint32_t pos1 = (uint32_t)(base + k) + 1u;
          // offsets exactly as the backward forms them, so both passes take the same decisions
          const float dx = fx - m.x;
          blend2<kCount, kClamp>(pp, q, c, dx, __fadd2_rn(fy, make_float2(-m.y, -m.y)), pos1);
        };
        if (cnt == kThreads) {  // a full batch: no bound checks
          for (int k0 = 0; k0 < kThreads; k0 += 8) {
#pragma unroll
            for (int u = 0; u < 8; ++u) one(k0 + u);
            if (pp.done0 && pp.done1) break;
          }
        } else {
          for (int k0 = 0; k0 < cnt; k0 += 4) {
#pragma unroll
            for (int u = 0; u < 4; ++u)
              if (k0 + u < cnt) one(k0 + u);
            if (pp.done0 && pp.done1) break;
          }
        }
      };
      if (!kCount && batch_no_clamp) run(std::false_type{});
      else run(std::true_type{});
    }
  }
  if (kCount) {
    unsigned long long e = (unsigned long long)pp.evaluated, c = (unsigned long long)pp.contributed;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      e += __shfl_xor_sync(0xffffffffu, e, o);
      c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    if (lane == 0 && e) atomicAdd(a.n_evaluated, e);
    if (lane == 0 && c) atomicAdd(a.n_evaluated + 1, c);
  }
  const float Ts[2] = {pp.T.x, pp.T.y};
  const float C0[2] = {pp.c0.x, pp.c0.y}, C1[2] = {pp.c1.x, pp.c1.y}, C2[2] = {pp.c2.x, pp.c2.y};
  const uint32_t lasts[2] = {pp.last0, pp.last1};
  const int rows[2] = {py0, py1};
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    if (px < a.width && rows[r] < a.height) {
      const int pix = rows[r] * a.width + px;
      a.image[3 * pix + 0] = C0[r] + Ts[r] * a.bg[0];
      a.image[3 * pix + 1] = C1[r] + Ts[r] * a.bg[1];
      a.image[3 * pix + 2] = C2[r] + Ts[r] * a.bg[2];
      a.final_T[pix] = Ts[r];
      a.n_contrib[pix] = lasts[r];
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
  a.n = (uint32_t)p.n;
  for (int c = 0; c < 3; ++c) a.bg[c] = v.bg[c];
  a.image = image;
  a.final_T = final_T;
  a.n_contrib = n_contrib;
  a.n_evaluated = reinterpret_cast<unsigned long long*>(n_evaluated);
  const int tiles = a.tiles_x * tiles_of(v.height);
  if (tiles == 0) return cudaSuccess;
  return launch_pdl(n_evaluated != nullptr ? render_fwd_kernel<true> : render_fwd_kernel<false>, dim3(tiles),
                    dim3(kThreads), 0, st, a);
}

}  // namespace sdgs
