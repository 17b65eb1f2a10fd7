// Backward pass: adjoint of compositing (per tile, back to front) and of the per-Gaussian
// geometry (SH colour, EWA projection, conic inverse, conditional slicing, modulation and
// Sigma = L L^T).  Discrete decisions (culling, radius, tile rectangles, per-pixel skips and the
// stop position) are those of the forward and carry no derivative.
#include "geometry.cuh"
#include "raster_common.cuh"

namespace sdgs {

namespace {

constexpr int kThreads = kTilePixels / 2;
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
  float bg[3];
  float* g2;  // [n][12]
};

// Sums g[0..8] over the warp by recursive halving: at each level a lane keeps one half of its
// values and adds its partner's copy of that half, so 16 exchanges replace 9 full butterflies.
// Afterwards lanes 2v and 2v + 1 hold the warp total of g[v] (v < 9); the result is returned
// for those lanes (and 0 for lanes whose v >= 9).
__device__ __forceinline__ float warp_sum9(const float g[9]) {
  const int lane = threadIdx.x & 31;
  float v[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = i < 9 ? g[i] : 0.f;
  // level k keeps the half of v selected by lane bit (4 - k) and folds the other half in
#pragma unroll
  for (int half = 8, bit = 16; half >= 1; half >>= 1, bit >>= 1) {
    const bool upper = (lane & bit) != 0;
#pragma unroll
    for (int i = 0; i < half; ++i) {
      const float send = upper ? v[i] : v[i + half];
      const float keep = upper ? v[i + half] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, bit);
    }
  }
  return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

// Per-pixel state of the back-to-front replay.
struct BwdPixel {
  float T;                 // transmittance in front of the current position
  float R0, R1, R2;        // colour seen behind the current position, normalised by T there
  float d0, d1, d2;        // dL/dC of the pixel
  uint32_t last;           // positions >= last were not blended in the forward
};

// Adjoint of one (pixel, Gaussian) blend for the thread's two pixels at once (rows r and r + 8:
// same dx, dy as a pair), without branches, accumulated into g[9] = d(u, v, a, b, c, alpha_cond,
// r, g, b).  A pixel that does not take the Gaussian gets alpha 0, which leaves its T, R and the
// gradient unchanged exactly; the decisions are those of the forward (same exponent, alpha and
// thresholds).  The gradient is accumulated per pixel in g2[9] (x: first pixel, y: second).
struct BwdPair {
  float2 T, R0, R1, R2, d0, d1, d2;
  uint32_t last0, last1;
};

__device__ __forceinline__ bool unblend2(BwdPair& px, const float4& co, const float4& q, const float4& c,
                                         float dx, float2 dy, uint32_t pos, float2 g[9]) {
  const float a = __fmul_rn(__fmul_rn(q.x, dx), dx);
  const float bx = __fmul_rn(q.y, dx);
  const float2 t = __ffma2_rn(make_float2(q.z, q.z), dy, make_float2(bx, bx));
  const float2 p2 = __ffma2_rn(dy, t, make_float2(a, a));
  const float2 G = make_float2(ex2_approx(p2.x), ex2_approx(p2.y));
  const float2 raw = __fmul2_rn(make_float2(co.w, co.w), G);
  const float2 al = make_float2(fminf(kAlphaMax, raw.x), fminf(kAlphaMax, raw.y));
  const bool h0 = pos < px.last0 && p2.x <= 0.f && al.x >= kAlphaMin;
  const bool h1 = pos < px.last1 && p2.y <= 0.f && al.y >= kAlphaMin;
  const float2 ae = make_float2(h0 ? al.x : 0.f, h1 ? al.y : 0.f);  // alpha taken (0: skipped)
  const float2 om = make_float2(1.f - ae.x, 1.f - ae.y);
  px.T = make_float2(__fdividef(px.T.x, om.x), __fdividef(px.T.y, om.y));
  const float2 w = __fmul2_rn(ae, px.T);
  g[6] = __ffma2_rn(px.d0, w, g[6]);
  g[7] = __ffma2_rn(px.d1, w, g[7]);
  g[8] = __ffma2_rn(px.d2, w, g[8]);
  float2 s = __fmul2_rn(px.d0, __fadd2_rn(make_float2(c.x, c.x), make_float2(-px.R0.x, -px.R0.y)));
  s = __ffma2_rn(px.d1, __fadd2_rn(make_float2(c.y, c.y), make_float2(-px.R1.x, -px.R1.y)), s);
  s = __ffma2_rn(px.d2, __fadd2_rn(make_float2(c.z, c.z), make_float2(-px.R2.x, -px.R2.y)), s);
  const float2 dal = __fmul2_rn(px.T, s);
  px.R0 = __ffma2_rn(om, px.R0, __fmul2_rn(make_float2(c.x, c.x), ae));
  px.R1 = __ffma2_rn(om, px.R1, __fmul2_rn(make_float2(c.y, c.y), ae));
  px.R2 = __ffma2_rn(om, px.R2, __fmul2_rn(make_float2(c.z, c.z), ae));
  // no derivative through the 0.99 clamp
  const float2 dl = make_float2(h0 && raw.x < kAlphaMax ? dal.x : 0.f, h1 && raw.y < kAlphaMax ? dal.y : 0.f);
  g[5] = __ffma2_rn(dl, make_float2(fminf(G.x, 1.f), fminf(G.y, 1.f)), g[5]);  // G <= 1 where taken
  const float2 dp = __fmul2_rn(dl, al);  // d alpha / d(power) = alpha
  const float2 ddx = __ffma2_rn(make_float2(co.y, co.y), dy, make_float2(co.x * dx, co.x * dx));
  const float2 ddy = __ffma2_rn(make_float2(co.z, co.z), dy, make_float2(co.y * dx, co.y * dx));
  g[0] = __ffma2_rn(dp, ddx, g[0]);
  g[1] = __ffma2_rn(dp, ddy, g[1]);
  const float hdx2 = -0.5f * dx * dx;
  g[2] = __ffma2_rn(dp, make_float2(hdx2, hdx2), g[2]);
  g[3] = __ffma2_rn(dp, __fmul2_rn(make_float2(-dx, -dx), dy), g[3]);
  g[4] = __ffma2_rn(dp, __fmul2_rn(make_float2(-0.5f, -0.5f), __fmul2_rn(dy, dy)), g[4]);
  return h0 || h1;
}

// Back-to-front replay per 16x16 tile, 128 threads with two pixels each (rows r and r + 8).
// The tile's list is staged from the back in batches of 128; each Gaussian's gradient is summed
// over the thread's pixels, then over the warp, and added to the per-Gaussian buffer with one
// atomic per component and warp.
__global__ void __launch_bounds__(kThreads) raster_bwd_kernel(const RasterBwdArgs a) {
  griddep_wait();
  __shared__ float2 s_xy[kThreads];
  __shared__ float4 s_co[kThreads];
  __shared__ float4 s_rgb[kThreads];
  __shared__ uint32_t s_id[kThreads];
  __shared__ float s_g[kThreads][9];  // this batch's per-Gaussian gradient, summed over the warps
  __shared__ uint32_t s_max;

  const int tile = blockIdx.x;
  const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
  const int lane = threadIdx.x & 31;
  const int px = tx * kTile + (threadIdx.x & (kTile - 1));
  const int py[2] = {ty * kTile + (int)(threadIdx.x / kTile), ty * kTile + (int)(threadIdx.x / kTile) + kTile / 2};
  const float fx = (float)px + 0.5f;
  const float fy[2] = {(float)py[0] + 0.5f, (float)py[1] + 0.5f};
  const uint2 range = a.ranges[tile];

  BwdPair pp;
  {
    BwdPixel pxs[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      BwdPixel& p = pxs[r];
      p.T = 1.f; p.last = 0; p.d0 = p.d1 = p.d2 = 0.f;
      p.R0 = a.bg[0]; p.R1 = a.bg[1]; p.R2 = a.bg[2];
      if (px < a.width && py[r] < a.height) {
        const int pix = py[r] * a.width + px;
        p.T = a.final_T[pix];
        p.last = a.n_contrib[pix];
        p.d0 = a.dL_dimage[3 * pix + 0];
        p.d1 = a.dL_dimage[3 * pix + 1];
        p.d2 = a.dL_dimage[3 * pix + 2];
      }
    }
    pp.T = make_float2(pxs[0].T, pxs[1].T);
    pp.R0 = make_float2(pxs[0].R0, pxs[1].R0);
    pp.R1 = make_float2(pxs[0].R1, pxs[1].R1);
    pp.R2 = make_float2(pxs[0].R2, pxs[1].R2);
    pp.d0 = make_float2(pxs[0].d0, pxs[1].d0);
    pp.d1 = make_float2(pxs[0].d1, pxs[1].d1);
    pp.d2 = make_float2(pxs[0].d2, pxs[1].d2);
    pp.last0 = pxs[0].last;
    pp.last1 = pxs[1].last;
  }
  const uint32_t mylast = max(pp.last0, pp.last1);
  const float2 fy2 = make_float2(fy[0], fy[1]);
  if (threadIdx.x == 0) s_max = 0;
  __syncthreads();
  atomicMax(&s_max, mylast);
  __syncthreads();
  const int end = (int)s_max;  // positions >= end were blended at no pixel of the tile

  for (int i = threadIdx.x; i < kThreads * 9; i += kThreads) (&s_g[0][0])[i] = 0.f;
  for (int top = end; top > 0; top -= kThreads) {
    const int lo = max(0, top - kThreads);
    const int j = lo + threadIdx.x;
    __syncthreads();  // the previous batch is fully consumed
    if (j < top) {
      const uint32_t gid = a.point_list[range.x + j];
      s_xy[threadIdx.x] = a.mean2d[gid];
      s_co[threadIdx.x] = a.conic_opacity[gid];
      s_rgb[threadIdx.x] = make_float4(a.rgb[3 * gid + 0], a.rgb[3 * gid + 1], a.rgb[3 * gid + 2], 0.f);
      s_id[threadIdx.x] = gid;
    }
    const int cnt = top - lo;
    __syncthreads();
    for (int k = cnt - 1; k >= 0; --k) {
      const float2 m = s_xy[k];
      const float4 co_k = s_co[k];
      const float4 q = scaled_conic(co_k);
      const float4 c = s_rgb[k];
      const uint32_t pos = (uint32_t)(lo + k);
      float2 g2[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) g2[i] = make_float2(0.f, 0.f);
      const float dx = fx - m.x;
      const bool hit = unblend2(pp, co_k, q, c, dx, __fadd2_rn(fy2, make_float2(-m.y, -m.y)), pos, g2);
      if (__any_sync(0xffffffffu, hit)) {
        float g[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) g[i] = g2[i].x + g2[i].y;
        const float tot = warp_sum9(g);
        const int v = lane >> 1;
        if ((lane & 1) == 0 && v < 9) atomicAdd(&s_g[k][v], tot);
      }
    }
    __syncthreads();
    // one set of global atomics per Gaussian and block
    if (threadIdx.x < cnt) {
      float* out = a.g2 + (size_t)kG2 * s_id[threadIdx.x];
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        const float x = s_g[threadIdx.x][i];
        if (x != 0.f) atomicAdd(out + i, x);
        s_g[threadIdx.x][i] = 0.f;
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
};

// For X = Lw^-1 Y with Lw lower triangular n x n (n = 3 or 4), given dX returns dY = Lw^-T dX.
template <int N>
__device__ __forceinline__ void solve_upper_T(const float Lw[N][N], const float dX[N], float dY[N]) {
#pragma unroll
  for (int i = N - 1; i >= 0; --i) {
    float s = dX[i];
#pragma unroll
    for (int k = i + 1; k < N; ++k) s -= Lw[k][i] * dY[k];
    dY[i] = s / Lw[i][i];
  }
}

// One visible Gaussian's adjoint; returns its d/d(lambda_t, lambda_d) in *dlt, *dld.
__device__ __forceinline__ void geom_bwd_one(const GeomBwdArgs& a, int64_t i, float* dlt, float* dld);

__global__ void __launch_bounds__(128, 3) geom_bwd_kernel(const GeomBwdArgs a) {
  const int64_t i = (int64_t)blockIdx.x * 128 + threadIdx.x;
  float dlt = 0.f, dld = 0.f;
  if (i < a.n) {
    const ushort4 rc = a.rect[i];
    if (rc.z > rc.x && rc.w > rc.y) geom_bwd_one(a, i, &dlt, &dld);
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
    const float rn = 1.f / sqrtf(w0 * w0 + w1 * w1 + w2 * w2);
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
      float4 d = dshp[q];
      d.x += Y[(4 * q) / 3] * dc[(4 * q) % 3];
      d.y += Y[(4 * q + 1) / 3] * dc[(4 * q + 1) % 3];
      d.z += Y[(4 * q + 2) / 3] * dc[(4 * q + 2) % 3];
      d.w += Y[(4 * q + 3) / 3] * dc[(4 * q + 3) % 3];
      dshp[q] = d;
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
  const float id2 = 1.f / (ps.det * ps.det);
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
    const float z = ps.p[2], rz = 1.f / z;
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
    a.dopacity[i] += dalc * ft * fd;
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
  for (int q = 0; q < 7; ++q) {
    float4 d = dLp[q];
    d.x += dLg[4 * q]; d.y += dLg[4 * q + 1]; d.z += dLg[4 * q + 2]; d.w += dLg[4 * q + 3];
    dLp[q] = d;
  }
#pragma unroll
  for (int k = 0; k < 7; ++k) a.dmean7[7 * i + k] += dm[k];
}

}  // namespace

size_t bwd_workspace_bytes(int64_t n) { return ((size_t)n * kG2 * sizeof(float) + 255) & ~size_t(255); }

cudaError_t launch_render_bwd(const sdgs_scene& s, const sdgs_view& v, const sdgs_projected& p,
                              const sdgs_bins& b, const float* final_T, const uint32_t* n_contrib,
                              const float* dL_dimage, char* ws, const sdgs_grads& g, cudaStream_t st) {
  if (s.n == 0) return cudaSuccess;
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
  r.width = v.width;
  r.height = v.height;
  r.tiles_x = tiles_of(v.width);
  for (int c = 0; c < 3; ++c) r.bg[c] = v.bg[c];
  r.g2 = g2;
  const int tiles = r.tiles_x * tiles_of(v.height);
  raster_bwd_kernel<<<tiles, kThreads, 0, st>>>(r);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  GeomBwdArgs a;
  a.mean7 = s.mean7; a.L28 = s.L28; a.opacity = s.opacity; a.sh = s.sh; a.n = s.n;
  a.q = make_query(s, v);
  a.cam = make_camera(v);
  a.rect = reinterpret_cast<const ushort4*>(p.rect);
  a.g2 = g2;
  a.dmean7 = g.dmean7; a.dL28 = g.dL28; a.dopacity = g.dopacity; a.dsh = g.dsh; a.dlambda = g.dlambda;
  geom_bwd_kernel<<<(unsigned)((s.n + 127) / 128), 128, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace sdgs
