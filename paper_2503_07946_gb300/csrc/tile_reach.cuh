// Which tiles of a Gaussian's rectangle it may reach (alpha >= 1/255 at some pixel centre): per tile
// row, one contiguous span of tiles.  Binning keeps a (tile, Gaussian) instance only inside the
// spans.
//
// The rule is conservative: every pixel centre of a dropped tile has alpha_cond exp(-q/2) < 1/255
// with a margin above FP32 error, so those pixels would skip the Gaussian anyway and the image does
// not change.  Because it decides which instances exist (an integer outcome), it is evaluated with
// correctly rounded operations only, in a fixed order, so that the same FP32 inputs always give the
// same spans.  With conic (a, b, c), opacity alpha and mean (u, v):
//   det = ac - b^2,  m = 1e-4 + 2^-18 (ac + b^2) / det   (relative FP32 error of the quadratic form)
//   lim = 512 (sqrt^8(255 alpha) - 1) + 1e-3              (>= 2 ln(255 alpha), ln y <= k (y^(1/k) - 1))
//   Q = lim (1 + 8m) / (1 - m): the ellipse {a dx^2 + 2b dx dy + c dy^2 <= Q} holds every pixel
//   centre with alpha >= 1/255.
//   hx = sqrt(Q c / det), hy = sqrt(Q a / det): its half extents; its rightmost point has
//   dy_r = (-b / c) hx and its leftmost -dy_r.
//   Row ty spans dy in [ey0, ey1] = [16 ty + 0.5 - v, 16 ty + 15.5 - v].  It is empty when the band
//   misses [-hy - pad_y, hy + pad_y].  Otherwise the ellipse's x-extent over the band (concave in
//   dy, so attained at the clamped dy_r and -dy_r) is
//     x_max = (-b d1 + sqrt(max(aQ - det d1^2, 0))) / a + pad_x,  d1 = clamp(dy_r, ey0, ey1)
//     x_min = (-b d2 - sqrt(max(aQ - det d2^2, 0))) / a - pad_x,  d2 = clamp(-dy_r, ey0, ey1)
//   with pad = 0.05 + 2e-3 h covering the FP32 error of the square roots near the ellipse's ends,
//   and the kept tiles are ceil((u + x_min - 15.5) / 16) <= tx <= floor((u + x_max - 0.5) / 16).
//   Everything is dropped when lim < 0 (alpha < 1/255); nothing when det <= 0, m >= 1/2, a <= 0
//   or lim is NaN.  A NaN bound keeps the whole row.
#pragma once

#include "common.cuh"

namespace sdgs {

struct SpanRule {
  float u, v, a, b, det, aQ, hx, reach_y, dyr, padx;
  int mode;  // 0: spans, 1: keep every tile of the rectangle, 2: drop every tile
};

__device__ __forceinline__ SpanRule span_setup(float2 xy, float4 co) {
  SpanRule r;
  r.u = xy.x; r.v = xy.y; r.a = co.x; r.b = co.y;
  const float a = co.x, b = co.y, c = co.z;
  const float ac = __fmul_rn(a, c), bb = __fmul_rn(b, b);
  const float det = __fsub_rn(ac, bb);
  r.det = det;
  const float m = __fadd_rn(1e-4f, __fmul_rn(3.814697265625e-06f, __fdiv_rn(__fadd_rn(ac, bb), det)));
  float y = __fmul_rn(255.f, co.w);
#pragma unroll
  for (int k = 0; k < 8; ++k) y = __fsqrt_rn(y);
  const float lim = __fadd_rn(__fmul_rn(512.f, __fsub_rn(y, 1.f)), 1e-3f);
  const bool never = !(det > 0.f) || !(m < 0.5f) || !(a > 0.f) || (lim != lim);
  r.mode = never ? 1 : (lim < 0.f ? 2 : 0);
  const float Q = __fdiv_rn(__fmul_rn(lim, __fadd_rn(1.f, __fmul_rn(8.f, m))), __fsub_rn(1.f, m));
  r.hx = __fsqrt_rn(__fdiv_rn(__fmul_rn(Q, c), det));
  const float hy = __fsqrt_rn(__fdiv_rn(__fmul_rn(Q, a), det));
  r.dyr = __fmul_rn(__fdiv_rn(-b, c), r.hx);
  r.padx = __fadd_rn(0.05f, __fmul_rn(2e-3f, r.hx));
  r.reach_y = __fadd_rn(hy, __fadd_rn(0.05f, __fmul_rn(2e-3f, hy)));
  r.aQ = __fmul_rn(a, Q);
  return r;
}

// The kept tiles [lo, hi] of row ty (mode 0); false when the row is empty.  lo / hi are integral
// floats and may be NaN (keep the row).
__device__ __forceinline__ bool span_row(const SpanRule& r, int ty, float* lo, float* hi) {
  const float y0 = __fadd_rn((float)(ty * kTile), 0.5f);
  const float ey0 = __fsub_rn(y0, r.v), ey1 = __fsub_rn(__fadd_rn(y0, 15.f), r.v);
  if (ey0 > r.reach_y || ey1 < -r.reach_y) return false;
  const float d1 = fminf(ey1, fmaxf(ey0, r.dyr));
  const float s1 = __fsqrt_rn(fmaxf(__fsub_rn(r.aQ, __fmul_rn(__fmul_rn(r.det, d1), d1)), 0.f));
  const float x_max = __fadd_rn(__fdiv_rn(__fadd_rn(-__fmul_rn(r.b, d1), s1), r.a), r.padx);
  const float d2 = fminf(ey1, fmaxf(ey0, -r.dyr));
  const float s2 = __fsqrt_rn(fmaxf(__fsub_rn(r.aQ, __fmul_rn(__fmul_rn(r.det, d2), d2)), 0.f));
  const float x_min = __fsub_rn(__fdiv_rn(__fsub_rn(-__fmul_rn(r.b, d2), s2), r.a), r.padx);
  // (x / 16 correctly rounded is x * 2^-4 correctly rounded: the same float, one multiply)
  *lo = ceilf(__fmul_rn(__fsub_rn(__fadd_rn(r.u, x_min), 15.5f), 0.0625f));
  *hi = floorf(__fmul_rn(__fsub_rn(__fadd_rn(r.u, x_max), 0.5f), 0.0625f));
  return true;
}

// Kept tiles [*x0, *x1) of row ty within the rectangle columns [rx0, rx1) (rx0 < rx1).
__device__ __forceinline__ void span_cols(const SpanRule& r, int ty, int rx0, int rx1, int* x0, int* x1) {
  if (r.mode == 1) { *x0 = rx0; *x1 = rx1; return; }
  float lo, hi;
  if (r.mode == 2 || !span_row(r, ty, &lo, &hi)) { *x0 = *x1 = rx0; return; }
  const float l = fmaxf(lo, (float)rx0), h = fminf(hi, (float)(rx1 - 1));  // NaN bound -> the edge
  if (!(h >= l)) { *x0 = *x1 = rx0; return; }
  *x0 = (int)l;
  *x1 = (int)h + 1;
}

// Rows that can hold a kept tile, a superset of the rows span_row accepts (so results never
// depend on it): the rectangle rows within one row of the band test's own limits.
__device__ __forceinline__ void span_rows(const SpanRule& r, int ry0, int ry1, int* y0, int* y1) {
  if (r.mode != 0) { *y0 = ry0; *y1 = r.mode == 1 ? ry1 : ry0; return; }
  const float inv = 1.f / kTile;
  const float t0 = floorf((r.v - r.reach_y - 15.5f) * inv) - 1.f;
  const float t1 = floorf((r.v + r.reach_y - 0.5f) * inv) + 2.f;
  if (!(t0 == t0) || !(t1 == t1)) { *y0 = ry0; *y1 = ry1; return; }
  *y0 = (int)fmaxf((float)ry0, fminf((float)ry1, t0));
  *y1 = (int)fmaxf((float)*y0, fminf((float)ry1, t1));
}

}  // namespace sdgs
