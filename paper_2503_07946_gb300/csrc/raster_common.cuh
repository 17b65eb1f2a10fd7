// Per-pixel opacity of one splat, shared by the forward and backward rasterisers.
//
// Both passes must take the same skip decision (alpha < 1/255) for every (pixel, Gaussian) pair,
// so the exponent and alpha are computed here with explicitly rounded operations (no
// compiler-chosen contraction) and the hardware ex2 instruction.
#pragma once

#include "common.cuh"

namespace sdgs {

constexpr float kNegHalfLog2e = -0.72134752044448170f;  // -log2(e) / 2
constexpr float kNegLog2e = -1.4426950408889634f;

// (a, b, c, alpha) of the conic -> coefficients of the exponent in log2 units:
// power2 = qa dx^2 + qb dx dy + qc dy^2 = log2(e) * (-(a dx^2 + c dy^2) / 2 - b dx dy)
__device__ __forceinline__ float4 scaled_conic(float4 co) {
  return make_float4(__fmul_rn(kNegHalfLog2e, co.x), __fmul_rn(kNegLog2e, co.y),
                     __fmul_rn(kNegHalfLog2e, co.z), co.w);
}

__device__ __forceinline__ float splat_power2(const float4& q, float dx, float dy) {
  const float a = __fmul_rn(__fmul_rn(q.x, dx), dx);
  const float t = __fmaf_rn(q.z, dy, __fmul_rn(q.y, dx));
  return __fmaf_rn(dy, t, a);
}

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Smallest exponent-argument a(x-u)^2 + 2b(x-u)(y-v) + c(y-v)^2 over the box [x0,x1] x [y0,y1]
// (zero when the mean lies inside).  On an edge the minimum over the free coordinate is at the
// clamped stationary point.  a, c > 0 for a positive-definite conic.  An approximate stationary
// point only raises the edge value by c (error)^2, a relative O(eps^2) far inside the margin of
// splat_misses_box.
__device__ __forceinline__ float conic_box_min(float a, float b, float c, float u, float v, float x0,
                                               float x1, float y0, float y1) {
  if (u >= x0 && u <= x1 && v >= y0 && v <= y1) return 0.f;
  float best = INFINITY;
  const float ex[2] = {x0 - u, x1 - u};
  const float ey[2] = {y0 - v, y1 - v};
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const float dx = ex[i];
    const float dy = fminf(ey[1], fmaxf(ey[0], __fdividef(-b * dx, c)));
    best = fminf(best, a * dx * dx + 2.f * b * dx * dy + c * dy * dy);
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const float dy = ey[i];
    const float dx = fminf(ex[1], fmaxf(ex[0], __fdividef(-b * dy, a)));
    best = fminf(best, a * dx * dx + 2.f * b * dx * dy + c * dy * dy);
  }
  return fmaxf(best, 0.f);
}

// True when alpha_cond exp(-q/2) < 1/255 at every pixel centre of the box, with a relative
// safety margin far above the FP32 rounding of either this test or the per-pixel evaluation.
// Both evaluate the quadratic form in FP32, whose relative error grows like
// eps (ac + b^2) / det for an elongated conic; the margin grows with it, and a conic too
// ill-conditioned for a margin below one half is never culled.
__device__ __forceinline__ bool splat_misses_box(float4 co, float2 xy, float x0, float x1, float y0,
                                                 float y1) {
  if (!(co.w >= kAlphaMin)) return true;
  const float ac = co.x * co.z, bb = co.y * co.y;
  const float det = ac - bb;
  if (!(det > 0.f)) return false;
  const float margin = 1e-4f + 64.f * 5.9604645e-8f * (ac + bb) / det;
  if (!(margin < 0.5f)) return false;
  const float thr = 2.f * __logf(255.f * co.w);  // q above this gives alpha < 1/255 (abs err ~1e-6)
  const float qmin = conic_box_min(co.x, co.y, co.z, xy.x, xy.y, x0, x1, y0, y1);
  return qmin * (1.f - margin) > thr + 1e-4f;
}

}  // namespace sdgs
