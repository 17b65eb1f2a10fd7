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

// A record whose conic is not positive definite (only caller-made records can be) is staged as
// conic 0 and opacity 0, so that every pixel skips it (exponent 0, alpha 0; with its own conic the
// exponent could overflow to +inf and 0 * inf make alpha NaN); the rasterisers then need no
// per-pixel sign test of the exponent.
__device__ __forceinline__ float4 pd_or_transparent(float4 co) {
  const bool pd = co.x > 0.f && __fsub_rn(__fmul_rn(co.x, co.z), __fmul_rn(co.y, co.y)) > 0.f;
  return pd ? co : make_float4(0.f, 0.f, 0.f, 0.f);
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

}  // namespace sdgs
