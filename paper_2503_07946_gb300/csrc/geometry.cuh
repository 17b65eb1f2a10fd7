// Per-Gaussian geometry of the 7DGS render path in FP32: conditional slicing (Sec. 4.2,
// Eqs. cond_mean / cond_cov, Algorithm 1 steps 3-5), modulation (Eqs. temp_mod / dir_mod,
// Algorithm 1 step 6), EWA projection and SH colour (Sec. 4.4, the 3DGS projection the paper
// adopts).  Used by the forward kernel and recomputed by the backward kernel.
//
// Slicing never forms Sigma = L L^T.  Forming it squares the conditioning of the (t, d) block,
// and FP32 then loses several digits of mu_cond for Gaussians whose query lies many standard
// deviations from their (t, d) mean.  Instead, the rows of L are reordered to (t, d | p) and
// the 7x7 matrix is made lower triangular again by Givens rotations of its columns (an
// orthogonal LQ step, backward stable):  P L Q = K,  so  K K^T = P Sigma P^T  with K the Cholesky
// factor of Sigma in the (t, d | p) order.  With K = [[K11, 0], [K21, K22]]:
//   mu_cond    = mu_p + K21 K11^-1 (x2 - mu2),   x2 = (t, d)     (= Eq. cond_mean)
//   Sigma_cond = K22 K22^T                                       (= Eq. cond_cov)
// since Sigma_(t,d) = K11 K11^T, Sigma_p,(t,d) = K21 K11^T and Sigma_p = K21 K21^T + K22 K22^T.
// Packed index of L[i][j] (j <= i) is i*(i+1)/2 + j.
#pragma once

#include "common.cuh"

namespace sdgs {

struct Camera {
  float R[3][3];
  float T[3];
  float fx, fy, cx, cy;
  float lim_x, lim_y;  // 1.3 tan(fov/2) along x and y
  float campos[3];
  float near_plane;
  int width, height, tiles_x, tiles_y;
};

struct Query {
  float t;
  float d[3];
  float lambda_t, lambda_d;
  int dir_mode;       // 1: d is each Gaussian's unit direction from campos to its mu_p
  float campos[3];
};

// The query Gaussian m is conditioned on: the request's, or with dir_mode = 1 its own
// direction d = (mu_p - campos) / |mu_p - campos|; *rn gets 1 / |mu_p - campos|.
__device__ __forceinline__ Query query_for(const Query& q, const float m[7], float* rn) {
  Query r = q;
  *rn = 0.f;
  if (q.dir_mode == 1) {
    const float w0 = m[0] - q.campos[0], w1 = m[1] - q.campos[1], w2 = m[2] - q.campos[2];
    const float inv = rsqrtf(w0 * w0 + w1 * w1 + w2 * w2);
    r.d[0] = w0 * inv; r.d[1] = w1 * inv; r.d[2] = w2 * inv;
    *rn = inv;
  }
  return r;
}

// Real SH constants of degree <= 3 (the standard Cartesian table, with the Condon-Shortley
// phase carried as the sign of the m != 0 entries).
__device__ __constant__ const float kSH0 = 0.28209479177387814f;
__device__ __constant__ const float kSH1 = 0.4886025119029199f;
__device__ __constant__ const float kSH2[5] = {1.0925484305920792f, -1.0925484305920792f,
                                              0.31539156525252005f, -1.0925484305920792f,
                                              0.5462742152960396f};
__device__ __constant__ const float kSH3[7] = {-0.5900435899266435f, 2.890611442640554f,
                                              -0.4570457994644658f, 0.3731763325901154f,
                                              -0.4570457994644658f, 1.445305721320277f,
                                              -0.5900435899266435f};

Camera make_camera(const sdgs_view& v);
Query make_query(const sdgs_scene& s, const sdgs_view& v);

// The 16 basis values at the unit direction (x, y, z).
__device__ __forceinline__ void sh_basis(float x, float y, float z, float Y[16]) {
  const float xx = x * x, yy = y * y, zz = z * z;
  Y[0] = kSH0;
  Y[1] = -kSH1 * y;
  Y[2] = kSH1 * z;
  Y[3] = -kSH1 * x;
  Y[4] = kSH2[0] * x * y;
  Y[5] = kSH2[1] * y * z;
  Y[6] = kSH2[2] * (2.f * zz - xx - yy);
  Y[7] = kSH2[3] * x * z;
  Y[8] = kSH2[4] * (xx - yy);
  Y[9] = kSH3[0] * y * (3.f * xx - yy);
  Y[10] = kSH3[1] * x * y * z;
  Y[11] = kSH3[2] * y * (4.f * zz - xx - yy);
  Y[12] = kSH3[3] * z * (2.f * zz - 3.f * xx - 3.f * yy);
  Y[13] = kSH3[4] * x * (4.f * zz - xx - yy);
  Y[14] = kSH3[5] * z * (xx - yy);
  Y[15] = kSH3[6] * x * (xx - 3.f * yy);
}

// Intermediate values of the forward that the backward needs again.
struct SliceState {
  float K11[4][4];  // Cholesky factor of Sigma_(t,d) (lower)
  float K21[3][4];  // Sigma_p,(t,d) K11^-T
  float A[3][3];    // K22: Sigma_cond = A A^T (lower)
  float v[4];       // K11^-1 (x2 - mu2)
  float mu[3];      // mu_cond
  // modulation
  float St;         // Sigma_t
  float C[3][3];    // Cholesky factor of Sigma_d (lower)
  float y[3];       // C^-1 (d - mu_d)
  float e_t, e_d;   // exponents of f_temp and f_dir
};

__device__ __forceinline__ float Lget(const float L[28], int i, int j) {
  return j <= i ? L[i * (i + 1) / 2 + j] : 0.f;
}

// Conditional slicing (Givens route above) and modulation for one Gaussian.
// L: packed 28 entries, m: mean7.  Returns alpha_cond.
__device__ __forceinline__ float slice_one(const float L[28], const float m[7], float alpha,
                                           const Query& q, SliceState& s) {
  // B = rows (t, dx, dy, dz, px, py, pz) of L
  float B[7][7];
#pragma unroll
  for (int r = 0; r < 7; ++r) {
    const int src = r < 4 ? r + 3 : r - 4;
#pragma unroll
    for (int c = 0; c < 7; ++c) B[r][c] = Lget(L, src, c);
  }
  // Zero the entries right of the diagonal, row by row, rotating column c into column r.
  // Rows above r are already zero in both columns and are left alone.
#pragma unroll
  for (int r = 0; r < 6; ++r) {
#pragma unroll
    for (int c = r + 1; c < 7; ++c) {
      if (r < 4 && c > r + 3) continue;  // structurally zero: the t, d rows of L end at column r + 3
      const float a = B[r][r], b = B[r][c];
      const float h2 = a * a + b * b;
      if (!(h2 > 0.f)) continue;
      const float ih = rsqrtf(h2);  // (a rotation off by a few ulp: far below the path's tolerance)
      const float cs = a * ih, sn = b * ih;
#pragma unroll
      for (int i = r; i < 7; ++i) {
        const float x = B[i][r], y = B[i][c];
        B[i][r] = cs * x + sn * y;
        B[i][c] = cs * y - sn * x;
      }
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) s.K11[i][j] = j <= i ? B[i][j] : 0.f;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
#pragma unroll
    for (int j = 0; j < 4; ++j) s.K21[i][j] = B[4 + i][j];
#pragma unroll
    for (int j = 0; j < 3; ++j) s.A[i][j] = j <= i ? B[4 + i][4 + j] : 0.f;
  }
  const float e[4] = {q.t - m[3], q.d[0] - m[4], q.d[1] - m[5], q.d[2] - m[6]};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    float acc = e[i];
#pragma unroll
    for (int j = 0; j < i; ++j) acc -= s.K11[i][j] * s.v[j];
    s.v[i] = __fdividef(acc, s.K11[i][i]);
  }
#pragma unroll
  for (int r = 0; r < 3; ++r)
    s.mu[r] = m[r] + s.K21[r][0] * s.v[0] + s.K21[r][1] * s.v[1] + s.K21[r][2] * s.v[2] +
              s.K21[r][3] * s.v[3];

  // Modulation with the marginal blocks: Sigma_t = |row 3 of L|^2, Sigma_d = rows 4..6 of L
  // times their transpose.
  s.St = L[6] * L[6] + L[7] * L[7] + L[8] * L[8] + L[9] * L[9];
  const float* r4 = L + 10;  // 5 entries
  const float* r5 = L + 15;  // 6 entries
  const float* r6 = L + 21;  // 7 entries
  float S44 = 0.f, S54 = 0.f, S64 = 0.f, S55 = 0.f, S65 = 0.f, S66 = 0.f;
#pragma unroll
  for (int k = 0; k < 5; ++k) { S44 += r4[k] * r4[k]; S54 += r5[k] * r4[k]; S64 += r6[k] * r4[k]; }
#pragma unroll
  for (int k = 0; k < 6; ++k) { S55 += r5[k] * r5[k]; S65 += r6[k] * r5[k]; }
#pragma unroll
  for (int k = 0; k < 7; ++k) S66 += r6[k] * r6[k];
  float (&C)[3][3] = s.C;
  // (square roots and their reciprocals from one approximate reciprocal square root each)
  const float ic0 = rsqrtf(S44);
  C[0][0] = S44 * ic0;
  C[1][0] = S54 * ic0;
  C[2][0] = S64 * ic0;
  const float p1 = S55 - C[1][0] * C[1][0];
  const float ic1 = rsqrtf(p1);
  C[1][1] = p1 * ic1;
  C[2][1] = (S65 - C[2][0] * C[1][0]) * ic1;
  const float p2 = S66 - C[2][0] * C[2][0] - C[2][1] * C[2][1];
  const float ic2 = rsqrtf(p2);
  C[2][2] = p2 * ic2;
  C[0][1] = C[0][2] = C[1][2] = 0.f;
  s.y[0] = e[1] * ic0;
  s.y[1] = (e[2] - C[1][0] * s.y[0]) * ic1;
  s.y[2] = (e[3] - C[2][0] * s.y[0] - C[2][1] * s.y[1]) * ic2;
  s.e_t = __fdividef(-0.5f * q.lambda_t * e[0] * e[0], s.St);
  s.e_d = -0.5f * q.lambda_d * (s.y[0] * s.y[0] + s.y[1] * s.y[1] + s.y[2] * s.y[2]);
  return alpha * expf(s.e_t) * expf(s.e_d);
}

struct ProjState {
  float p[3];      // camera-space mu_cond
  float txz, tyz;  // clamped x/z, y/z used in J
  bool clx, cly;   // clamp active
  float Tm[2][3];  // J R
  float B[2][3];   // J R A
  float cov[3];    // a, b, c of Sigma_2D (dilated)
  float det;
};

// EWA projection of (mu_cond, Sigma_cond = A A^T).  Returns false if culled by depth or det.
__device__ __forceinline__ bool project_one(const Camera& cam, const SliceState& s, ProjState& ps) {
#pragma unroll
  for (int r = 0; r < 3; ++r)
    ps.p[r] = cam.R[r][0] * s.mu[0] + cam.R[r][1] * s.mu[1] + cam.R[r][2] * s.mu[2] + cam.T[r];
  const float z = ps.p[2];
  if (!(z >= cam.near_plane)) return false;
  const float rz = __fdividef(1.f, z);
  const float xz = ps.p[0] * rz, yz = ps.p[1] * rz;
  ps.txz = fminf(cam.lim_x, fmaxf(-cam.lim_x, xz));
  ps.tyz = fminf(cam.lim_y, fmaxf(-cam.lim_y, yz));
  ps.clx = (xz != ps.txz);
  ps.cly = (yz != ps.tyz);
  // J = [[fx/z, 0, -fx txz / z], [0, fy/z, -fy tyz / z]];  Tm = J R
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    ps.Tm[0][j] = cam.fx * rz * (cam.R[0][j] - ps.txz * cam.R[2][j]);
    ps.Tm[1][j] = cam.fy * rz * (cam.R[1][j] - ps.tyz * cam.R[2][j]);
  }
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int k = 0; k < 3; ++k)
      ps.B[r][k] = ps.Tm[r][0] * s.A[0][k] + ps.Tm[r][1] * s.A[1][k] + ps.Tm[r][2] * s.A[2][k];
  ps.cov[0] = ps.B[0][0] * ps.B[0][0] + ps.B[0][1] * ps.B[0][1] + ps.B[0][2] * ps.B[0][2] + kDilation;
  ps.cov[1] = ps.B[0][0] * ps.B[1][0] + ps.B[0][1] * ps.B[1][1] + ps.B[0][2] * ps.B[1][2];
  ps.cov[2] = ps.B[1][0] * ps.B[1][0] + ps.B[1][1] * ps.B[1][1] + ps.B[1][2] * ps.B[1][2] + kDilation;
  ps.det = ps.cov[0] * ps.cov[2] - ps.cov[1] * ps.cov[1];
  return ps.det > 0.f;
}

}  // namespace sdgs
