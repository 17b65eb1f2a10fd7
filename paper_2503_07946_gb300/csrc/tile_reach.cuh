// Which tiles of a Gaussian's rectangle it may reach (alpha >= 1/255 at some pixel).  Binning keeps
// a (tile, Gaussian) instance only for those tiles.
//
// The rule is conservative: for a dropped tile, alpha_cond exp(-q/2) < 1/255 at every pixel centre
// with a margin far above FP32 error, so the pixels of that tile would skip the Gaussian anyway and
// the image does not change.  Because it decides which instances exist (an integer outcome), it is
// evaluated with correctly rounded operations only, in a fixed order, so that the same FP32
// inputs always give the same decision:
//   q_min  = min over the tile's pixel-centre box of a dx^2 + 2b dx dy + c dy^2: 0 if the mean is
//            inside; else the least of the (one or two) edges that face the mean -- the convex
//            form grows along any segment from the mean, and such a segment enters the box
//            through a facing edge -- each at its clamped stationary point
//            dy = clamp((-b / c) dx) or dx = clamp((-b / a) dy)
//   thr    = 512 (sqrt^8(255 alpha) - 1) >= 2 ln(255 alpha)      (ln y <= k (y^(1/k) - 1), k = 256)
//   m      = 1e-4 + 64 * 2^-24 (ac + b^2) / (ac - b^2)          (FP32 error of the quadratic form)
//   drop   iff  ac - b^2 > 0  and  m < 1/2  and  q_min (1 - m) > thr + 1e-3
#pragma once

#include "common.cuh"

namespace sdgs {

struct __align__(16) Reach {
  float u, v, a, b, c;
  float sx, sy;     // -b / c and -b / a: stationary points dy* = sx dx, dx* = sy dy
  float lim;        // thr + 1e-3
  float keep_frac;  // 1 - m
  float det;        // ac - b^2
  int never_drop;
  float pad;
};

__device__ __forceinline__ Reach reach_setup(float2 xy, float4 co) {
  Reach r;
  r.u = xy.x; r.v = xy.y; r.a = co.x; r.b = co.y; r.c = co.z;
  r.sx = __fdiv_rn(-co.y, co.z);
  r.sy = __fdiv_rn(-co.y, co.x);
  const float ac = __fmul_rn(co.x, co.z), bb = __fmul_rn(co.y, co.y);
  const float det = __fsub_rn(ac, bb);
  r.det = det;
  const float m = __fadd_rn(1e-4f, __fmul_rn(3.814697265625e-06f, __fdiv_rn(__fadd_rn(ac, bb), det)));
  float y = __fmul_rn(255.f, co.w);
#pragma unroll
  for (int k = 0; k < 8; ++k) y = __fsqrt_rn(y);
  const float thr = __fmul_rn(512.f, __fsub_rn(y, 1.f));
  r.lim = __fadd_rn(thr, 1e-3f);
  r.keep_frac = __fsub_rn(1.f, m);
  r.never_drop = !(det > 0.f) || !(m < 0.5f);
  return r;
}

__device__ __forceinline__ float reach_q(const Reach& r, float dx, float dy) {
  return __fadd_rn(__fadd_rn(__fmul_rn(__fmul_rn(r.a, dx), dx), __fmul_rn(__fmul_rn(__fmul_rn(2.f, r.b), dx), dy)),
                   __fmul_rn(__fmul_rn(r.c, dy), dy));
}

__device__ __forceinline__ bool reach_tile(const Reach& r, int tx, int ty) {
  if (r.never_drop) return true;
  const float x0 = __fadd_rn((float)(tx * kTile), 0.5f), x1 = __fadd_rn(x0, 15.f);
  const float y0 = __fadd_rn((float)(ty * kTile), 0.5f), y1 = __fadd_rn(y0, 15.f);
  const bool lo_x = r.u < x0, hi_x = r.u > x1, lo_y = r.v < y0, hi_y = r.v > y1;
  const bool facing_x = lo_x || hi_x, facing_y = lo_y || hi_y;
  if (!facing_x && !facing_y) return !(0.f > r.lim);  // mean inside the box: q_min = 0
  const float ex0 = __fsub_rn(x0, r.u), ex1 = __fsub_rn(x1, r.u);
  const float ey0 = __fsub_rn(y0, r.v), ey1 = __fsub_rn(y1, r.v);
  float best = INFINITY;
  if (facing_x) {
    const float dx = lo_x ? ex0 : ex1;
    best = reach_q(r, dx, fminf(ey1, fmaxf(ey0, __fmul_rn(r.sx, dx))));
  }
  if (facing_y) {
    const float dy = lo_y ? ey0 : ey1;
    best = fminf(best, reach_q(r, fminf(ex1, fmaxf(ex0, __fmul_rn(r.sy, dy))), dy));
  }
  return !(__fmul_rn(fmaxf(best, 0.f), r.keep_frac) > r.lim);
}

// Tiles of `rect` that can contain a reachable pixel box: the rectangle clipped to a bounding box
// of the ellipse {q <= (1.02 + m) (thr + 1e-3) / (1 - m)}, plus 2% + 1 px.  The FP32 error of the
// quadratic form in reach_tile is below ~0.1 m relative, so every tile it keeps lies inside (the
// kept set is defined over the full rectangle; this only skips tiles that cannot pass, so results
// never depend on it).  Ordinary FP32 is fine here.
__device__ __forceinline__ ushort4 reach_bounds(const Reach& r, ushort4 rect) {
  if (r.never_drop || r.lim != r.lim) return rect;
  if (r.lim < 0.f) return make_ushort4(rect.x, rect.y, rect.x, rect.y);  // no pixel can reach
  const float m = 1.f - r.keep_frac;
  const float Q = (1.02f + m) * r.lim / r.keep_frac;
  const float hx = 1.02f * sqrtf(Q * r.c / r.det) + 1.f;
  const float hy = 1.02f * sqrtf(Q * r.a / r.det) + 1.f;
  if (!(hx < 1e9f) || !(hy < 1e9f)) return rect;
  const float inv = 1.f / kTile;
  const float x0 = floorf((r.u - hx - 16.f) * inv), x1 = floorf((r.u + hx) * inv) + 1.f;
  const float y0 = floorf((r.v - hy - 16.f) * inv), y1 = floorf((r.v + hy) * inv) + 1.f;
  ushort4 o = rect;
  o.x = (unsigned short)fmaxf((float)rect.x, fminf((float)rect.z, x0));
  o.z = (unsigned short)fmaxf((float)o.x, fminf((float)rect.z, x1));
  o.y = (unsigned short)fmaxf((float)rect.y, fminf((float)rect.w, y0));
  o.w = (unsigned short)fmaxf((float)o.y, fminf((float)rect.w, y1));
  return o;
}

}  // namespace sdgs
