// Backward pass: adjoint of compositing (per tile, back to front) and of the per-Gaussian
// geometry (SH colour, EWA projection, conic inverse, conditional slicing, modulation and
// Sigma = L L^T).  Discrete decisions (culling, radius, tile rectangles, per-pixel skips and the
// stop position) are those of the forward and carry no derivative.
#include "geometry.cuh"
#include "raster_common.cuh"

namespace sdgs {

namespace {

constexpr int kThreads = kTilePixels;
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

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

__global__ void __launch_bounds__(kThreads) raster_bwd_kernel(const RasterBwdArgs a) {
  __shared__ float2 s_xy[kThreads];
  __shared__ float4 s_co[kThreads];  // a, b, c, alpha_cond
  __shared__ float s_rgb[3][kThreads];
  __shared__ uint32_t s_id[kThreads];
  __shared__ uint32_t s_max;

  const int tile = blockIdx.x;
  const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
  const int px = tx * kTile + (threadIdx.x & (kTile - 1));
  const int py = ty * kTile + (threadIdx.x / kTile);
  const bool inside = px < a.width && py < a.height;
  const int pix = py * a.width + px;
  const float fx = (float)px + 0.5f, fy = (float)py + 0.5f;
  const uint2 range = a.ranges[tile];

  float T = 1.f, dL0 = 0.f, dL1 = 0.f, dL2 = 0.f;
  uint32_t last = 0;
  if (inside) {
    T = a.final_T[pix];
    last = a.n_contrib[pix];
    dL0 = a.dL_dimage[3 * pix + 0];
    dL1 = a.dL_dimage[3 * pix + 1];
    dL2 = a.dL_dimage[3 * pix + 2];
  }
  // colour seen behind the current position, normalised by the transmittance there
  float R0 = a.bg[0], R1 = a.bg[1], R2 = a.bg[2];

  if (threadIdx.x == 0) s_max = 0;
  __syncthreads();
  atomicMax(&s_max, last);
  __syncthreads();
  const int end = (int)s_max;  // positions >= end contribute to no pixel of the tile

  for (int top = end; top > 0; top -= kThreads) {
    const int lo = max(0, top - kThreads);
    const int j = lo + threadIdx.x;
    __syncthreads();
    if (j < top) {
      const uint32_t g = a.point_list[range.x + j];
      s_id[threadIdx.x] = g;
      s_xy[threadIdx.x] = a.mean2d[g];
      s_co[threadIdx.x] = a.conic_opacity[g];
      s_rgb[0][threadIdx.x] = a.rgb[3 * g + 0];
      s_rgb[1][threadIdx.x] = a.rgb[3 * g + 1];
      s_rgb[2][threadIdx.x] = a.rgb[3 * g + 2];
    }
    __syncthreads();
    for (int k = top - lo - 1; k >= 0; --k) {
      const int pos = lo + k;  // position in the tile list
      float gu = 0.f, gv = 0.f, ga = 0.f, gb = 0.f, gc = 0.f, gal = 0.f, gr = 0.f, gg = 0.f, gbl = 0.f;
      bool contrib = false;
      if ((uint32_t)pos < last) {
        const float2 xy = s_xy[k];
        const float4 q = s_co[k];
        const float dx = fx - xy.x, dy = fy - xy.y;
        // identical arithmetic to the forward so that the skip decisions agree
        const float p2 = splat_power2(scaled_conic(q), dx, dy);
        if (p2 <= 0.f) {
          const float G = ex2_approx(p2);
          const float raw = __fmul_rn(q.w, G);
          const float al = fminf(kAlphaMax, raw);
          if (al >= kAlphaMin) {
            contrib = true;
            T = T / (1.f - al);
            const float c0 = s_rgb[0][k], c1 = s_rgb[1][k], c2 = s_rgb[2][k];
            const float w = al * T;
            gr = dL0 * w; gg = dL1 * w; gbl = dL2 * w;
            const float dal = T * (dL0 * (c0 - R0) + dL1 * (c1 - R1) + dL2 * (c2 - R2));
            R0 = c0 * al + (1.f - al) * R0;
            R1 = c1 * al + (1.f - al) * R1;
            R2 = c2 * al + (1.f - al) * R2;
            if (raw < kAlphaMax) {
              gal = dal * G;
              const float dp = dal * al;  // d alpha / d power = alpha
              gu = dp * (q.x * dx + q.y * dy);
              gv = dp * (q.y * dx + q.z * dy);
              ga = -0.5f * dp * dx * dx;
              gb = -dp * dx * dy;
              gc = -0.5f * dp * dy * dy;
            }
          }
        }
      }
      if (__any_sync(0xffffffffu, contrib)) {
        gu = warp_sum(gu); gv = warp_sum(gv); ga = warp_sum(ga); gb = warp_sum(gb); gc = warp_sum(gc);
        gal = warp_sum(gal); gr = warp_sum(gr); gg = warp_sum(gg); gbl = warp_sum(gbl);
        if ((threadIdx.x & 31) == 0) {
          float* out = a.g2 + (size_t)kG2 * s_id[k];
          atomicAdd(out + 0, gu); atomicAdd(out + 1, gv); atomicAdd(out + 2, ga); atomicAdd(out + 3, gb);
          atomicAdd(out + 4, gc); atomicAdd(out + 5, gal); atomicAdd(out + 6, gr); atomicAdd(out + 7, gg);
          atomicAdd(out + 8, gbl);
        }
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

__global__ void __launch_bounds__(128) geom_bwd_kernel(const GeomBwdArgs a) {
  const int64_t i = (int64_t)blockIdx.x * 128 + threadIdx.x;
  if (i >= a.n) return;
  const ushort4 rc = a.rect[i];
  if (!(rc.z > rc.x && rc.w > rc.y)) return;

  float L[28];
#pragma unroll
  for (int k = 0; k < 28; ++k) L[k] = a.L28[28 * i + k];
  float m[7];
#pragma unroll
  for (int k = 0; k < 7; ++k) m[k] = a.mean7[7 * i + k];
  const float alpha = a.opacity[i];
  const float* gp = a.g2 + (size_t)kG2 * i;
  const float du = gp[0], dv = gp[1], dA_ = gp[2], dB_ = gp[3], dC_ = gp[4], dalc = gp[5];
  const float drgb[3] = {gp[6], gp[7], gp[8]};

  SliceState s;
  const float alpha_c = slice_one(L, m, alpha, a.q, s);
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
    const float* shp = a.sh + 48 * i;
    float raw[3] = {0.5f, 0.5f, 0.5f};
#pragma unroll
    for (int k = 0; k < 16; ++k)
#pragma unroll
      for (int c = 0; c < 3; ++c) raw[c] += Y[k] * shp[3 * k + c];
    float dc[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) dc[c] = raw[c] > 0.f ? drgb[c] : 0.f;
    float dY[16];
    float* dshp = a.dsh + 48 * i;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      dY[k] = 0.f;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        dshp[3 * k + c] += Y[k] * dc[c];
        dY[k] += shp[3 * k + c] * dc[c];
      }
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
  // cov = P P^T + 0.3 I with P = Tm A (2x3)
  float dP[2][3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    dP[0][k] = 2.f * da * ps.B[0][k] + db * ps.B[1][k];
    dP[1][k] = db * ps.B[0][k] + 2.f * dc * ps.B[1][k];
  }
  float dA[3][3], dTm[2][3];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int k = 0; k < 3; ++k) dA[r][k] = ps.Tm[0][r] * dP[0][k] + ps.Tm[1][r] * dP[1][k];
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int j = 0; j < 3; ++j) dTm[r][j] = dP[r][0] * s.A[j][0] + dP[r][1] * s.A[j][1] + dP[r][2] * s.A[j][2];

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

  // ---- mu_cond = mu_p + A z ----
  float dz[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    dm[k] += dmu[k];
    dz[k] = s.A[0][k] * dmu[0] + s.A[1][k] * dmu[1] + s.A[2][k] * dmu[2];
#pragma unroll
    for (int r = 0; r < 3; ++r) dA[r][k] += dmu[r] * s.z[k];
  }

  // ---- A = L11 H^-T (A^T = H^-1 L11^T) and z = H^-1 u ----
  float dH[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
  float dL11[3][3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {  // column r of A^T is row r of A
    float dX[3] = {dA[r][0], dA[r][1], dA[r][2]}, dY[3];
    solve_upper_T<3>(s.H, dX, dY);
#pragma unroll
    for (int k = 0; k < 3; ++k) dL11[r][k] = dY[k];
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
      for (int q2 = 0; q2 <= p; ++q2) dH[p][q2] -= dY[p] * s.A[r][q2];
  }
  float du3[3];
  solve_upper_T<3>(s.H, dz, du3);
#pragma unroll
  for (int p = 0; p < 3; ++p)
#pragma unroll
    for (int q2 = 0; q2 <= p; ++q2) dH[p][q2] -= du3[p] * s.z[q2];
  dLg[0] += dL11[0][0];
  dLg[1] += dL11[1][0]; dLg[2] += dL11[1][1];
  dLg[3] += dL11[2][0]; dLg[4] += dL11[2][1]; dLg[5] += dL11[2][2];

  // ---- H = chol(G), reverse of the scalar recurrences ----
  float dG[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
  {
    const float (&H)[3][3] = s.H;
    float h00 = dH[0][0], h10 = dH[1][0], h20 = dH[2][0], h11 = dH[1][1], h21 = dH[2][1], h22 = dH[2][2];
    const float s22 = h22 / (2.f * H[2][2]);
    dG[2][2] = s22; h20 += -2.f * H[2][0] * s22; h21 += -2.f * H[2][1] * s22;
    dG[2][1] = h21 / H[1][1]; h20 += -H[1][0] * h21 / H[1][1]; h10 += -H[2][0] * h21 / H[1][1];
    h11 += -H[2][1] * h21 / H[1][1];
    const float s11 = h11 / (2.f * H[1][1]);
    dG[1][1] = s11; h10 += -2.f * H[1][0] * s11;
    dG[2][0] = h20 / H[0][0]; h00 += -H[2][0] * h20 / H[0][0];
    dG[1][0] = h10 / H[0][0]; h00 += -H[1][0] * h10 / H[0][0];
    dG[0][0] = h00 / (2.f * H[0][0]);
  }
  // ---- G = I + M^T M (lower entries), u = M^T v ----
  float dM[4][3], dv4[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    dv4[r] = s.M[r][0] * du3[0] + s.M[r][1] * du3[1] + s.M[r][2] * du3[2];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float acc = du3[c] * s.v[r];
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const float gab = (c >= b) ? dG[c][b] : dG[b][c];
        acc += gab * s.M[r][b] * (c == b ? 2.f : 1.f);
      }
      dM[r][c] = acc;
    }
  }
  // ---- M = L22^-1 L21, v = L22^-1 e ----
  const float L22[4][4] = {{L[9], 0.f, 0.f, 0.f}, {L[13], L[14], 0.f, 0.f},
                           {L[18], L[19], L[20], 0.f}, {L[24], L[25], L[26], L[27]}};
  float dL22[4][4] = {{0.f}};
  const int iL21[4][3] = {{6, 7, 8}, {10, 11, 12}, {15, 16, 17}, {21, 22, 23}};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float dX[4] = {dM[0][c], dM[1][c], dM[2][c], dM[3][c]}, dY[4];
    solve_upper_T<4>(L22, dX, dY);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      dLg[iL21[r][c]] += dY[r];
#pragma unroll
      for (int q2 = 0; q2 <= r; ++q2) dL22[r][q2] -= dY[r] * s.M[q2][c];
    }
  }
  {
    float de[4];
    solve_upper_T<4>(L22, dv4, de);
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int q2 = 0; q2 <= r; ++q2) dL22[r][q2] -= de[r] * s.v[q2];
    dm[3] -= de[0]; dm[4] -= de[1]; dm[5] -= de[2]; dm[6] -= de[3];
  }
  dLg[9] += dL22[0][0];
  dLg[13] += dL22[1][0]; dLg[14] += dL22[1][1];
  dLg[18] += dL22[2][0]; dLg[19] += dL22[2][1]; dLg[20] += dL22[2][2];
  dLg[24] += dL22[3][0]; dLg[25] += dL22[3][1]; dLg[26] += dL22[3][2]; dLg[27] += dL22[3][3];

  // ---- alpha_cond = alpha exp(e_t) exp(e_d) ----
  {
    const float ft = expf(s.e_t), fd = expf(s.e_d);
    a.dopacity[i] += dalc * ft * fd;
    const float de_ = dalc * alpha_c;  // d alpha_c / d e_t = d alpha_c / d e_d = alpha_c
    const float e0 = a.q.t - m[3];
    // e_t = -1/2 lambda_t e0^2 / S_t
    dm[3] += de_ * a.q.lambda_t * e0 / s.St;
    const float dSt = de_ * 0.5f * a.q.lambda_t * e0 * e0 / (s.St * s.St);
#pragma unroll
    for (int k = 0; k < 4; ++k) dLg[6 + k] += 2.f * dSt * L[6 + k];
    // e_d = -1/2 lambda_d q, q = delta^T Sigma_d^-1 delta = |y|^2, y = C^-1 delta
    const float dq = -0.5f * a.q.lambda_d * de_;
    float w[3];
    solve_upper_T<3>(s.C, s.y, w);  // w = C^-T y = Sigma_d^-1 delta
#pragma unroll
    for (int k = 0; k < 3; ++k) dm[4 + k] -= 2.f * dq * w[k];
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

#pragma unroll
  for (int k = 0; k < 28; ++k) a.dL28[28 * i + k] += dLg[k];
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
  a.dmean7 = g.dmean7; a.dL28 = g.dL28; a.dopacity = g.dopacity; a.dsh = g.dsh;
  geom_bwd_kernel<<<(unsigned)((s.n + 127) / 128), 128, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace sdgs
