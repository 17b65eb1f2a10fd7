// Backward pass: adjoint of compositing (per tile, back to front) and of the per-Gaussian
// geometry (SH colour, EWA projection, conic inverse, conditional slicing, modulation and
// Sigma = L L^T).  Discrete decisions (culling, radius, tile rectangles, per-pixel skips and the
// stop position) are those of the forward and carry no derivative.
#include "geometry.cuh"
#include "raster_common.cuh"

namespace sdgs {

namespace {

constexpr int kG2 = 12;  // floats per Gaussian of screen-space gradient: u v a b c alpha r g b _ _ _

struct RasterBwdArgs {
  const float2* mean2d;
  const float4* conic_opacity;
  const float* rgb;
  const uint32_t* point_list;
  const uint2* ranges;
  const float* final_T;
  const uint32_t* n_contrib;
  const float* dL_dimage;
  int width, height, tiles_x;
  uint32_t n;  // Gaussians in the records; a list entry >= n (never written by binning) is skipped
  float bg[3];
  float* g2;  // [n][12]
};

// Sums g[0..8] over the warp.  g[0..7] by recursive halving over lane bits 16, 8 and 4 (at each
// level a lane keeps one half of its values and adds its partner's copy of that half), g[8] by
// butterflies over the same bits; then the pair (g[c], g[8]) is halved over bit 2 and summed over
// bit 1: 12 exchanges.  Afterwards a lane with bit 2 clear holds the warp total of
// g[(lane >> 2) & 7] and a lane with bit 2 set the total of g[8].
__device__ __forceinline__ float warp_sum9(const float g[9]) {
  const int lane = threadIdx.x & 31;
  float v[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = g[i];
  float e = g[8];
#pragma unroll
  for (int half = 4, bit = 16; half >= 1; half >>= 1, bit >>= 1) {
    const bool upper = (lane & bit) != 0;
#pragma unroll
    for (int i = 0; i < half; ++i) {
      const float send = upper ? v[i] : v[i + half];
      const float keep = upper ? v[i + half] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, bit);
    }
    e += __shfl_xor_sync(0xffffffffu, e, bit);
  }
  const bool upper = (lane & 2) != 0;
  const float keep = upper ? e : v[0];
  const float x = keep + __shfl_xor_sync(0xffffffffu, upper ? v[0] : e, 2);
  return x + __shfl_xor_sync(0xffffffffu, x, 1);
}

// Per-pixel state of the back-to-front replay for a pair of a thread's pixels (one column, the
// same dx): transmittance in front of the current position, DR = dL/dC . R with R the colour seen
// behind the current position normalised by T there, dL/dC, and the forward's stop position
// (positions >= last were not blended).
struct BwdPair {
  float2 T, DR, d0, d1, d2;
  uint32_t last0, last1;
};

// Adjoint of one (pixel, Gaussian) blend for both pixels, without branches.  A pixel that does not
// take the Gaussian gets alpha 0, which leaves T, DR and the sums unchanged exactly; the decisions
// are those of the forward (same exponent, alpha and thresholds).  With dl = dL/d alpha (0 where
// not taken or where the 0.99 clamp was active) and G the Gaussian's value, it accumulates, per
// pixel (x: first, y: second),
//   g = (dlG dx, dlG dy, dlG dx^2, dlG dx dy, dlG dy^2, dlG, dL/dr, dL/dg, dL/db),  dlG = dl G,
// from which the flush forms d(u, v, a, b, c) with the conic and alpha_cond (alpha = alpha_cond G,
// d alpha / d power = alpha) and d alpha_cond = sum dlG.  q is the scaled conic with q.w =
// alpha_cond.
__device__ __forceinline__ bool unblend2(BwdPair& px, const float4& q, const float4& c, float dx, float2 dy,
                                         uint32_t pos, float2 g[9]) {
  const float a = __fmul_rn(__fmul_rn(q.x, dx), dx);
  const float bx = __fmul_rn(q.y, dx);
  const float2 t = __ffma2_rn(make_float2(q.z, q.z), dy, make_float2(bx, bx));
  const float2 p2 = __ffma2_rn(dy, t, make_float2(a, a));
  const float2 G = make_float2(ex2_approx(p2.x), ex2_approx(p2.y));
  const float2 raw = __fmul2_rn(make_float2(q.w, q.w), G);
  const float2 al = make_float2(fminf(kAlphaMax, raw.x), fminf(kAlphaMax, raw.y));
  const bool h0 = pos < px.last0 && al.x >= kAlphaMin;
  const bool h1 = pos < px.last1 && al.y >= kAlphaMin;
  const float2 ae = make_float2(h0 ? al.x : 0.f, h1 ? al.y : 0.f);  // alpha taken (0: skipped)
  const float2 om = make_float2(1.f - ae.x, 1.f - ae.y);
  px.T = make_float2(__fdividef(px.T.x, om.x), __fdividef(px.T.y, om.y));
  const float2 w = __fmul2_rn(ae, px.T);
  g[6] = __ffma2_rn(px.d0, w, g[6]);
  g[7] = __ffma2_rn(px.d1, w, g[7]);
  g[8] = __ffma2_rn(px.d2, w, g[8]);
  // dL/dC . c, then dL/d alpha = T (dL/dC . c - DR) and DR <- (1 - alpha) DR + alpha dL/dC . c
  float2 dc = __fmul2_rn(px.d0, make_float2(c.x, c.x));
  dc = __ffma2_rn(px.d1, make_float2(c.y, c.y), dc);
  dc = __ffma2_rn(px.d2, make_float2(c.z, c.z), dc);
  const float2 dal = __fmul2_rn(px.T, __fadd2_rn(dc, make_float2(-px.DR.x, -px.DR.y)));
  px.DR = __ffma2_rn(ae, dc, __fmul2_rn(om, px.DR));
  // no derivative through the 0.99 clamp
  const float2 dl = make_float2(h0 && raw.x < kAlphaMax ? dal.x : 0.f, h1 && raw.y < kAlphaMax ? dal.y : 0.f);
  const float2 dlG = __fmul2_rn(dl, G);
  g[5] = __fadd2_rn(g[5], dlG);
  const float2 dx2 = make_float2(dx, dx);
  g[0] = __ffma2_rn(dlG, dx2, g[0]);
  g[1] = __ffma2_rn(dlG, dy, g[1]);
  const float dxx = dx * dx;
  g[2] = __ffma2_rn(dlG, make_float2(dxx, dxx), g[2]);
  g[3] = __ffma2_rn(dlG, __fmul2_rn(dx2, dy), g[3]);
  g[4] = __ffma2_rn(dlG, __fmul2_rn(dy, dy), g[4]);
  return h0 || h1;
}

constexpr int kBwdThreads = kTilePixels / 4;
constexpr int kBatch = 128;

// The pixel state of a pair (rows py0 and py1 of column px) from the forward's outputs.
__device__ __forceinline__ void load_pair(const RasterBwdArgs& a, int px, int py0, int py1, BwdPair& pp) {
  float T[2], DR[2], d[2][3];
  uint32_t last[2];
  const int py[2] = {py0, py1};
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    T[r] = 1.f; last[r] = 0; d[r][0] = d[r][1] = d[r][2] = 0.f;
    if (px < a.width && py[r] < a.height) {
      const int pix = py[r] * a.width + px;
      T[r] = a.final_T[pix];
      last[r] = a.n_contrib[pix];
      d[r][0] = a.dL_dimage[3 * pix + 0];
      d[r][1] = a.dL_dimage[3 * pix + 1];
      d[r][2] = a.dL_dimage[3 * pix + 2];
    }
    DR[r] = d[r][0] * a.bg[0] + d[r][1] * a.bg[1] + d[r][2] * a.bg[2];  // R = background at the end
  }
  pp.T = make_float2(T[0], T[1]);
  pp.DR = make_float2(DR[0], DR[1]);
  pp.d0 = make_float2(d[0][0], d[1][0]);
  pp.d1 = make_float2(d[0][1], d[1][1]);
  pp.d2 = make_float2(d[0][2], d[1][2]);
  pp.last0 = last[0];
  pp.last1 = last[1];
}

// Back-to-front replay per 16x16 tile, 64 threads with four pixels each: column x, rows r, r + 8
// (pair A) and r + 4, r + 12 (pair B).  The tile's list is staged from the back in batches of 128;
// each Gaussian's sums are added over the thread's pixels, then over the warp, then over the
// block's warps in shared memory, and the batch ends with one set of global atomics per Gaussian.
__global__ void __launch_bounds__(kBwdThreads, 16) raster_bwd_kernel(const RasterBwdArgs a) {
  griddep_wait();
  __shared__ float2 s_xy[kBatch];
  __shared__ float4 s_co[kBatch];  // conic and alpha_cond
  __shared__ float4 s_q[kBatch];   // scaled conic and alpha_cond
  __shared__ float4 s_rgb[kBatch];
  __shared__ uint32_t s_id[kBatch];
  __shared__ float s_g[kBatch][9];  // this batch's per-Gaussian sums over the tile
  __shared__ uint32_t s_max;

  const int tile = blockIdx.x;
  const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
  const int lane = threadIdx.x & 31;
  const int px = tx * kTile + (threadIdx.x & (kTile - 1));
  const int r0 = ty * kTile + (int)(threadIdx.x / kTile);
  const float fx = (float)px + 0.5f;
  const uint2 range = a.ranges[tile];

  BwdPair pa, pb;
  load_pair(a, px, r0, r0 + 8, pa);
  load_pair(a, px, r0 + 4, r0 + 12, pb);
  const uint32_t mylast = max(max(pa.last0, pa.last1), max(pb.last0, pb.last1));
  const float2 fya = make_float2((float)r0 + 0.5f, (float)(r0 + 8) + 0.5f);
  const float2 fyb = make_float2((float)(r0 + 4) + 0.5f, (float)(r0 + 12) + 0.5f);
  if (threadIdx.x == 0) s_max = 0;
  __syncthreads();
  atomicMax(&s_max, mylast);
  __syncthreads();
  const int end = (int)s_max;  // positions >= end were blended at no pixel of the tile

  // the lane that adds a warp total into s_g, and which sum it holds
  const bool adder = (lane & 3) == 0 || lane == 2;
  const int slot = (lane & 2) ? 8 : (lane >> 2);
  for (int i = threadIdx.x; i < kBatch * 9; i += kBwdThreads) (&s_g[0][0])[i] = 0.f;
  for (int top = end; top > 0; top -= kBatch) {
    const int lo = max(0, top - kBatch);
    __syncthreads();  // the previous batch is fully consumed
#pragma unroll
    for (int h = 0; h < kBatch / kBwdThreads; ++h) {
      const int e = threadIdx.x + h * kBwdThreads;
      const int j = lo + e;
      if (j < top) {
        const uint32_t gid = a.point_list[range.x + j];
        const bool ok = gid < a.n;
        const float4 co = ok ? pd_or_transparent(a.conic_opacity[gid]) : make_float4(0.f, 0.f, 0.f, 0.f);
        s_xy[e] = ok ? a.mean2d[gid] : make_float2(0.f, 0.f);
        s_co[e] = co;
        s_q[e] = scaled_conic(co);
        s_rgb[e] = ok ? make_float4(a.rgb[3 * gid + 0], a.rgb[3 * gid + 1], a.rgb[3 * gid + 2], 0.f)
                      : make_float4(0.f, 0.f, 0.f, 0.f);
        s_id[e] = ok ? gid : 0xffffffffu;
      }
    }
    const int cnt = top - lo;
    __syncthreads();
    for (int k = cnt - 1; k >= 0; --k) {
      const float2 m = s_xy[k];
      const float4 q = s_q[k];
      const float4 c = s_rgb[k];
      const uint32_t pos = (uint32_t)(lo + k);
      float2 g2[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) g2[i] = make_float2(0.f, 0.f);
      const float dx = fx - m.x;
      const float2 my = make_float2(-m.y, -m.y);
      const bool ha = unblend2(pa, q, c, dx, __fadd2_rn(fya, my), pos, g2);
      const bool hb = unblend2(pb, q, c, dx, __fadd2_rn(fyb, my), pos, g2);
      if (__any_sync(0xffffffffu, ha || hb)) {
        float g[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) g[i] = g2[i].x + g2[i].y;
        const float tot = warp_sum9(g);
        if (adder) atomicAdd(&s_g[k][slot], tot);
      }
    }
    __syncthreads();
    // one set of global atomics per Gaussian and block: d(u, v) = alpha_cond Conic (Sx, Sy),
    // d(a, b, c) = -alpha_cond (Sxx / 2, Sxy, Syy / 2)
    for (int e = threadIdx.x; e < cnt; e += kBwdThreads) {
      if (s_id[e] == 0xffffffffu) continue;  // a skipped entry gathered nothing
      float* out = a.g2 + (size_t)kG2 * s_id[e];
      const float4 co = s_co[e];
      float* S = s_g[e];
      const float al = co.w;
      float o[9];
      o[0] = al * (co.x * S[0] + co.y * S[1]);
      o[1] = al * (co.y * S[0] + co.z * S[1]);
      o[2] = -0.5f * al * S[2];
      o[3] = -al * S[3];
      o[4] = -0.5f * al * S[4];
#pragma unroll
      for (int i = 5; i < 9; ++i) o[i] = S[i];
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        if (o[i] != 0.f) atomicAdd(out + i, o[i]);
        S[i] = 0.f;
      }
    }
  }
}

struct GeomBwdArgs {
  const float* mean7;
  const float* L28;
  const float* opacity;
  const float* sh;
  int64_t n;
  Query q;
  Camera cam;
  const ushort4* rect;
  const float* g2;
  float* dmean7;
  float* dL28;
  float* dopacity;
  float* dsh;
  float* dlambda;  // [2] or NULL
  bool overwrite;  // write the gradients (zero for culled Gaussians) instead of adding to them
};

__device__ __forceinline__ void put_grad(const GeomBwdArgs& a, float* p, float v) {
  if (a.overwrite) *p = v;
  else atomicAdd(p, v);
}
__device__ __forceinline__ void put_grad4(const GeomBwdArgs& a, float4* p, float4 v) {
  if (a.overwrite) *p = v;
  else atomicAdd(p, v);
}

// For X = Lw^-1 Y with Lw lower triangular n x n (n = 3 or 4), given dX returns dY = Lw^-T dX.
template <int N>
__device__ __forceinline__ void solve_upper_T(const float Lw[N][N], const float dX[N], float dY[N]) {
#pragma unroll
  for (int i = N - 1; i >= 0; --i) {
    float s = dX[i];
#pragma unroll
    for (int k = i + 1; k < N; ++k) s -= Lw[k][i] * dY[k];
    dY[i] = __fdividef(s, Lw[i][i]);
  }
}

// One visible Gaussian's adjoint; returns its d/d(lambda_t, lambda_d) in *dlt, *dld.
__device__ __forceinline__ void geom_bwd_one(const GeomBwdArgs& a, int64_t i, float* dlt, float* dld);

__global__ void __launch_bounds__(128, 3) geom_bwd_kernel(const GeomBwdArgs a) {
  const int64_t i = (int64_t)blockIdx.x * 128 + threadIdx.x;
  float dlt = 0.f, dld = 0.f;
  if (i < a.n) {
    const ushort4 rc = a.rect[i];
    if (rc.z > rc.x && rc.w > rc.y) {
      geom_bwd_one(a, i, &dlt, &dld);
    } else if (a.overwrite) {  // a culled Gaussian: zero gradients
      const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
      float4* dLp = reinterpret_cast<float4*>(a.dL28 + 28 * i);
#pragma unroll
      for (int q = 0; q < 7; ++q) dLp[q] = z;
      float4* dshp = reinterpret_cast<float4*>(a.dsh + 48 * i);
#pragma unroll
      for (int q = 0; q < 12; ++q) dshp[q] = z;
#pragma unroll
      for (int k = 0; k < 7; ++k) a.dmean7[7 * i + k] = 0.f;
      a.dopacity[i] = 0.f;
    }
  }
  if (a.dlambda == nullptr) return;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    dlt += __shfl_xor_sync(0xffffffffu, dlt, o);
    dld += __shfl_xor_sync(0xffffffffu, dld, o);
  }
  if ((threadIdx.x & 31) == 0 && (dlt != 0.f || dld != 0.f)) {
    atomicAdd(a.dlambda, dlt);
    atomicAdd(a.dlambda + 1, dld);
  }
}

__device__ __forceinline__ void geom_bwd_one(const GeomBwdArgs& a, int64_t i, float* dlt, float* dld) {

  float L[28];
  const float4* Lp = reinterpret_cast<const float4*>(a.L28 + 28 * i);  // 112-byte rows: aligned
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    const float4 v = __ldg(Lp + k);
    L[4 * k] = v.x; L[4 * k + 1] = v.y; L[4 * k + 2] = v.z; L[4 * k + 3] = v.w;
  }
  float m[7];
#pragma unroll
  for (int k = 0; k < 7; ++k) m[k] = __ldg(a.mean7 + 7 * i + k);
  const float alpha = a.opacity[i];
  const float* gp = a.g2 + (size_t)kG2 * i;
  const float du = gp[0], dv = gp[1], dA_ = gp[2], dB_ = gp[3], dC_ = gp[4], dalc = gp[5];
  const float drgb[3] = {gp[6], gp[7], gp[8]};

  SliceState s;
  float rnd;
  const Query q = query_for(a.q, m, &rnd);
  const float alpha_c = slice_one(L, m, alpha, q, s);
  ProjState ps;
  project_one(a.cam, s, ps);
  const Camera& cam = a.cam;

  float dmu[3] = {0.f, 0.f, 0.f};  // d mu_cond
  float dLg[28];
#pragma unroll
  for (int k = 0; k < 28; ++k) dLg[k] = 0.f;
  float dm[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};

  // ---- SH colour ----
  {
    float w0 = s.mu[0] - cam.campos[0], w1 = s.mu[1] - cam.campos[1], w2 = s.mu[2] - cam.campos[2];
    const float rn = rsqrtf(w0 * w0 + w1 * w1 + w2 * w2);
    const float x = w0 * rn, y = w1 * rn, z = w2 * rn;
    float Y[16];
    sh_basis(x, y, z, Y);
    // 192-byte SH rows (and their gradients) as 12 float4: flat index f = 3 k + c
    const float4* shp = reinterpret_cast<const float4*>(a.sh + 48 * i);
    float raw[3] = {0.5f, 0.5f, 0.5f};
#pragma unroll
    for (int q = 0; q < 12; ++q) {
      const float4 v = __ldg(shp + q);
      raw[(4 * q) % 3] += Y[(4 * q) / 3] * v.x;
      raw[(4 * q + 1) % 3] += Y[(4 * q + 1) / 3] * v.y;
      raw[(4 * q + 2) % 3] += Y[(4 * q + 2) / 3] * v.z;
      raw[(4 * q + 3) % 3] += Y[(4 * q + 3) / 3] * v.w;
    }
    float dc[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) dc[c] = raw[c] > 0.f ? drgb[c] : 0.f;
    float dY[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) dY[k] = 0.f;
    float4* dshp = reinterpret_cast<float4*>(a.dsh + 48 * i);
#pragma unroll
    for (int q = 0; q < 12; ++q) {
      const float4 v = __ldg(shp + q);  // second read: L1
      dY[(4 * q) / 3] += v.x * dc[(4 * q) % 3];
      dY[(4 * q + 1) / 3] += v.y * dc[(4 * q + 1) % 3];
      dY[(4 * q + 2) / 3] += v.z * dc[(4 * q + 2) % 3];
      dY[(4 * q + 3) / 3] += v.w * dc[(4 * q + 3) % 3];
      put_grad4(a, dshp + q, make_float4(Y[(4 * q) / 3] * dc[(4 * q) % 3], Y[(4 * q + 1) / 3] * dc[(4 * q + 1) % 3],
                                      Y[(4 * q + 2) / 3] * dc[(4 * q + 2) % 3],
                                      Y[(4 * q + 3) / 3] * dc[(4 * q + 3) % 3]));
    }
    const float xx = x * x, yy = y * y, zz = z * z;
    float gx = 0.f, gy = 0.f, gz = 0.f;
    gy += -kSH1 * dY[1];
    gz += kSH1 * dY[2];
    gx += -kSH1 * dY[3];
    gx += kSH2[0] * y * dY[4]; gy += kSH2[0] * x * dY[4];
    gy += kSH2[1] * z * dY[5]; gz += kSH2[1] * y * dY[5];
    gx += -2.f * kSH2[2] * x * dY[6]; gy += -2.f * kSH2[2] * y * dY[6]; gz += 4.f * kSH2[2] * z * dY[6];
    gx += kSH2[3] * z * dY[7]; gz += kSH2[3] * x * dY[7];
    gx += 2.f * kSH2[4] * x * dY[8]; gy += -2.f * kSH2[4] * y * dY[8];
    gx += 6.f * kSH3[0] * x * y * dY[9]; gy += kSH3[0] * (3.f * xx - 3.f * yy) * dY[9];
    gx += kSH3[1] * y * z * dY[10]; gy += kSH3[1] * x * z * dY[10]; gz += kSH3[1] * x * y * dY[10];
    gx += -2.f * kSH3[2] * x * y * dY[11]; gy += kSH3[2] * (4.f * zz - xx - 3.f * yy) * dY[11];
    gz += 8.f * kSH3[2] * y * z * dY[11];
    gx += -6.f * kSH3[3] * x * z * dY[12]; gy += -6.f * kSH3[3] * y * z * dY[12];
    gz += kSH3[3] * (6.f * zz - 3.f * xx - 3.f * yy) * dY[12];
    gx += kSH3[4] * (4.f * zz - 3.f * xx - yy) * dY[13]; gy += -2.f * kSH3[4] * x * y * dY[13];
    gz += 8.f * kSH3[4] * x * z * dY[13];
    gx += 2.f * kSH3[5] * x * z * dY[14]; gy += -2.f * kSH3[5] * y * z * dY[14];
    gz += kSH3[5] * (xx - yy) * dY[14];
    gx += kSH3[6] * (3.f * xx - 3.f * yy) * dY[15]; gy += -6.f * kSH3[6] * x * y * dY[15];
    // through dir = w / |w|
    const float dot = gx * x + gy * y + gz * z;
    dmu[0] += (gx - dot * x) * rn;
    dmu[1] += (gy - dot * y) * rn;
    dmu[2] += (gz - dot * z) * rn;
  }

  // ---- conic = inverse of the 2D covariance ----
  const float ca = ps.cov[0], cb = ps.cov[1], cc = ps.cov[2];
  const float id2 = __fdividef(1.f, ps.det * ps.det);
  const float da = (-cc * cc * dA_ + cb * cc * dB_ - cb * cb * dC_) * id2;
  const float db = (2.f * cb * cc * dA_ - (ca * cc + cb * cb) * dB_ + 2.f * ca * cb * dC_) * id2;
  const float dc = (-cb * cb * dA_ + ca * cb * dB_ - ca * ca * dC_) * id2;
  // cov = Tm Sigma_cond Tm^T + 0.3 I with Sigma_cond = A A^T: gradients w.r.t. Sigma_cond (as a
  // symmetric matrix) and w.r.t. Tm
  float Sc[3][3];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int k = 0; k < 3; ++k) Sc[r][k] = s.A[r][0] * s.A[k][0] + s.A[r][1] * s.A[k][1] + s.A[r][2] * s.A[k][2];
  const float* T0 = ps.Tm[0];
  const float* T1 = ps.Tm[1];
  float dS[3][3];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int k = 0; k < 3; ++k)
      dS[r][k] = da * T0[r] * T0[k] + 0.5f * db * (T0[r] * T1[k] + T1[r] * T0[k]) + dc * T1[r] * T1[k];
  float dTm[2][3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const float s0 = Sc[j][0] * T0[0] + Sc[j][1] * T0[1] + Sc[j][2] * T0[2];
    const float s1 = Sc[j][0] * T1[0] + Sc[j][1] * T1[1] + Sc[j][2] * T1[2];
    dTm[0][j] = 2.f * da * s0 + db * s1;
    dTm[1][j] = db * s0 + 2.f * dc * s1;
  }

  // ---- Tm = J R and the projected mean ----
  {
    const float z = ps.p[2], rz = __fdividef(1.f, z);
    float drz = 0.f, dtx = 0.f, dty = 0.f;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      drz += dTm[0][j] * cam.fx * (cam.R[0][j] - ps.txz * cam.R[2][j]) +
             dTm[1][j] * cam.fy * (cam.R[1][j] - ps.tyz * cam.R[2][j]);
      dtx += -cam.fx * rz * cam.R[2][j] * dTm[0][j];
      dty += -cam.fy * rz * cam.R[2][j] * dTm[1][j];
    }
    float dp[3] = {0.f, 0.f, 0.f};
    if (!ps.clx) { dp[0] += dtx * rz; drz += dtx * ps.p[0]; }
    if (!ps.cly) { dp[1] += dty * rz; drz += dty * ps.p[1]; }
    dp[0] += du * cam.fx * rz;
    dp[1] += dv * cam.fy * rz;
    drz += du * cam.fx * ps.p[0] + dv * cam.fy * ps.p[1];
    dp[2] += -drz * rz * rz;
#pragma unroll
    for (int k = 0; k < 3; ++k) dmu[k] += cam.R[0][k] * dp[0] + cam.R[1][k] * dp[1] + cam.R[2][k] * dp[2];
  }

  // ---- conditioning: mu_cond = mu_p + B W e,  Sigma_cond = Sigma_p - B W B^T ----
  // with B = Sigma_p,(t,d), W = Sigma_(t,d)^-1, e = (t - mu_t, d - mu_d), evaluated through the
  // stable factor of the forward: H = W B^T = K11^-T K21^T, w = W e = K11^-T v.
  float Hm[4][3], w4[4];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float h[4];
    solve_upper_T<4>(s.K11, s.K21[c], h);
#pragma unroll
    for (int k = 0; k < 4; ++k) Hm[k][c] = h[k];
  }
  solve_upper_T<4>(s.K11, s.v, w4);
  float Hd[4];  // H dmu = d e (the gradient w.r.t. e)
#pragma unroll
  for (int k = 0; k < 4; ++k) Hd[k] = Hm[k][0] * dmu[0] + Hm[k][1] * dmu[1] + Hm[k][2] * dmu[2];
#pragma unroll
  for (int k = 0; k < 3; ++k) dm[k] += dmu[k];
#pragma unroll
  for (int k = 0; k < 4; ++k) dm[3 + k] -= Hd[k];
  float ded[3] = {Hd[1], Hd[2], Hd[3]};  // gradient w.r.t. the conditioning direction d
  // G: gradient w.r.t. the symmetric 7x7 Sigma (order p, t, d), then dL = 2 G L.
  float G[7][7];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int k = 0; k < 3; ++k) G[r][k] = dS[r][k];
  float SH[3][4];  // dS H^T
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int k = 0; k < 4; ++k) SH[r][k] = dS[r][0] * Hm[k][0] + dS[r][1] * Hm[k][1] + dS[r][2] * Hm[k][2];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float dB = dmu[r] * w4[k] - 2.f * SH[r][k];
      G[r][3 + k] = 0.5f * dB;
      G[3 + k][r] = 0.5f * dB;
    }
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int l = 0; l < 4; ++l)
      G[3 + k][3 + l] = Hm[k][0] * SH[0][l] + Hm[k][1] * SH[1][l] + Hm[k][2] * SH[2][l] -
                        0.5f * (Hd[k] * w4[l] + w4[k] * Hd[l]);
#pragma unroll
  for (int i2 = 0; i2 < 7; ++i2)
#pragma unroll
    for (int j = 0; j <= i2; ++j) {
      float acc = 0.f;
#pragma unroll
      for (int k = j; k < 7; ++k) acc += G[i2][k] * Lget(L, k, j);
      dLg[i2 * (i2 + 1) / 2 + j] += 2.f * acc;
    }

  // ---- alpha_cond = alpha exp(e_t) exp(e_d) ----
  {
    const float ft = expf(s.e_t), fd = expf(s.e_d);
    put_grad(a, a.dopacity + i, dalc * ft * fd);
    const float de_ = dalc * alpha_c;  // d alpha_c / d e_t = d alpha_c / d e_d = alpha_c
    const float e0 = q.t - m[3];
    // e_t = -1/2 lambda_t e0^2 / S_t
    dm[3] += de_ * q.lambda_t * e0 / s.St;
    *dlt = de_ * (-0.5f * e0 * e0 / s.St);
    const float dSt = de_ * 0.5f * q.lambda_t * e0 * e0 / (s.St * s.St);
#pragma unroll
    for (int k = 0; k < 4; ++k) dLg[6 + k] += 2.f * dSt * L[6 + k];
    // e_d = -1/2 lambda_d q, q = delta^T Sigma_d^-1 delta = |y|^2, y = C^-1 delta
    const float dq = -0.5f * q.lambda_d * de_;
    *dld = de_ * (-0.5f * (s.y[0] * s.y[0] + s.y[1] * s.y[1] + s.y[2] * s.y[2]));
    float w[3];
    solve_upper_T<3>(s.C, s.y, w);  // w = C^-T y = Sigma_d^-1 delta
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      dm[4 + k] -= 2.f * dq * w[k];
      ded[k] += 2.f * dq * w[k];
    }
    // d Sigma_d = -dq w w^T; d L_d = 2 dSigma_d L_d on the stored (lower) entries of rows 4..6
    const int row0[3] = {10, 15, 21};
    const int len[3] = {5, 6, 7};
#pragma unroll
    for (int ra = 0; ra < 3; ++ra) {
#pragma unroll
      for (int k = 0; k < 7; ++k) {
        if (k >= len[ra]) break;
        float acc = 0.f;
#pragma unroll
        for (int rb = 0; rb < 3; ++rb)
          if (k < len[rb]) acc += w[rb] * L[row0[rb] + k];
        dLg[row0[ra] + k] += -2.f * dq * w[ra] * acc;
      }
    }
  }

  // ---- d = (mu_p - campos) / |mu_p - campos| (dir_mode = 1): dmu_p += (I - d d^T) ded / |w| ----
  if (q.dir_mode == 1) {
    const float dot = ded[0] * q.d[0] + ded[1] * q.d[1] + ded[2] * q.d[2];
#pragma unroll
    for (int k = 0; k < 3; ++k) dm[k] += (ded[k] - dot * q.d[k]) * rnd;
  }

  float4* dLp = reinterpret_cast<float4*>(a.dL28 + 28 * i);
#pragma unroll
  for (int q = 0; q < 7; ++q) put_grad4(a, dLp + q, make_float4(dLg[4 * q], dLg[4 * q + 1], dLg[4 * q + 2], dLg[4 * q + 3]));
#pragma unroll
  for (int k = 0; k < 7; ++k) put_grad(a, a.dmean7 + 7 * i + k, dm[k]);
}

}  // namespace

size_t bwd_workspace_bytes(int64_t n) { return ((size_t)n * kG2 * sizeof(float) + 255) & ~size_t(255); }

cudaError_t launch_render_bwd(const sdgs_scene& s, const sdgs_view& v, const sdgs_projected& p,
                              const sdgs_bins& b, const float* final_T, const uint32_t* n_contrib,
                              const float* dL_dimage, char* ws, const sdgs_grads& g, cudaStream_t st) {
  if (s.n == 0) {
    if (g.overwrite != 0 && g.dlambda != nullptr) return cudaMemsetAsync(g.dlambda, 0, 2 * sizeof(float), st);
    return cudaSuccess;
  }
  float* g2 = reinterpret_cast<float*>(ws);
  cudaError_t e = cudaMemsetAsync(g2, 0, (size_t)s.n * kG2 * sizeof(float), st);
  if (e != cudaSuccess) return e;
  RasterBwdArgs r;
  r.mean2d = reinterpret_cast<const float2*>(p.mean2d);
  r.conic_opacity = reinterpret_cast<const float4*>(p.conic_opacity);
  r.rgb = p.rgb;
  r.point_list = b.point_list;
  r.ranges = reinterpret_cast<const uint2*>(b.ranges);
  r.final_T = final_T;
  r.n_contrib = n_contrib;
  r.dL_dimage = dL_dimage;
  r.n = (uint32_t)p.n;
  r.width = v.width;
  r.height = v.height;
  r.tiles_x = tiles_of(v.width);
  for (int c = 0; c < 3; ++c) r.bg[c] = v.bg[c];
  r.g2 = g2;
  const int tiles = r.tiles_x * tiles_of(v.height);
  raster_bwd_kernel<<<tiles, kBwdThreads, 0, st>>>(r);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  GeomBwdArgs a;
  a.mean7 = s.mean7; a.L28 = s.L28; a.opacity = s.opacity; a.sh = s.sh; a.n = s.n;
  a.q = make_query(s, v);
  a.cam = make_camera(v);
  a.rect = reinterpret_cast<const ushort4*>(p.rect);
  a.g2 = g2;
  a.dmean7 = g.dmean7; a.dL28 = g.dL28; a.dopacity = g.dopacity; a.dsh = g.dsh; a.dlambda = g.dlambda;
  a.overwrite = g.overwrite != 0;
  if (a.overwrite && a.dlambda != nullptr) {  // (summed over the Gaussians by atomics)
    e = cudaMemsetAsync(a.dlambda, 0, 2 * sizeof(float), st);
    if (e != cudaSuccess) return e;
  }
  geom_bwd_kernel<<<(unsigned)((s.n + 127) / 128), 128, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace sdgs
