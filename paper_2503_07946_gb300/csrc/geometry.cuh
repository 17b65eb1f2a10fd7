// Per-Gaussian geometry of the 7DGS render path in FP32: conditional slicing (Sec. 4.2,
// Eqs. cond_mean / cond_cov, Algorithm 1 steps 3-5), modulation (Eqs. temp_mod / dir_mod,
// Algorithm 1 step 6), EWA projection and SH colour (Sec. 4.3, the 3DGS projection the paper
// adopts).  Used by the forward kernel and recomputed by the backward kernel.
//
// Slicing is evaluated through the precision form of the Schur complement instead of the
// literal Sigma_p - Sigma_p,(t,d) Sigma_(t,d)^-1 Sigma_p,(t,d)^T, which cancels badly in FP32
// when the conditional is much narrower than Sigma_p.  With L = [[L11, 0], [L21, L22]]
// (block 1 = p, block 2 = (t, d)) and M = L22^-1 L21 (4x3):
//   Sigma_cond = L11 G^-1 L11^T,  G = I + M^T M      (eigenvalues >= 1)
//   mu_cond    = mu_p + L11 G^-1 M^T L22^-1 (x2 - mu2),  x2 = (t, d)
// which equal Eqs. cond_cov / cond_mean exactly (Sigma_12 = L11 M^T L22^T,
// Sigma_22 = L22 (M M^T + I) L22^T and the push-through identity).  With G = H H^T (Cholesky):
//   A = L11 H^-T,  Sigma_cond = A A^T,  mu_cond = mu_p + A H^-1 M^T v,  v = L22^-1 (x2 - mu2).
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
};

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
  // M = L22^-1 L21 (rows r = t, dx, dy, dz; cols = p.x, p.y, p.z), v = L22^-1 (x2 - mu2)
  float M[4][3];
  float v[4];
  float H[3][3];  // Cholesky factor of G = I + M^T M (lower)
  float z[3];     // H^-1 M^T v
  float A[3][3];  // L11 H^-T
  float mu[3];    // mu_cond
  // modulation
  float St;       // Sigma_t
  float C[3][3];  // Cholesky factor of Sigma_d (lower)
  float y[3];     // C^-1 (d - mu_d)
  float e_t, e_d; // exponents of f_temp and f_dir
};

// Conditional slicing (precision form above) and modulation for one Gaussian.
// L: packed 28 entries, m: mean7.  Returns alpha_cond.
__device__ __forceinline__ float slice_one(const float L[28], const float m[7], float alpha,
                                           const Query& q, SliceState& s) {
  // L21 rows (t, dx, dy, dz) x cols (p.x, p.y, p.z); L22 lower 4x4.
  const float L21[4][3] = {{L[6], L[7], L[8]}, {L[10], L[11], L[12]},
                           {L[15], L[16], L[17]}, {L[21], L[22], L[23]}};
  const float d0 = 1.f / L[9], d1 = 1.f / L[14], d2 = 1.f / L[20], d3 = 1.f / L[27];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float m0 = L21[0][c] * d0;
    const float m1 = (L21[1][c] - L[13] * m0) * d1;
    const float m2 = (L21[2][c] - L[18] * m0 - L[19] * m1) * d2;
    const float m3 = (L21[3][c] - L[24] * m0 - L[25] * m1 - L[26] * m2) * d3;
    s.M[0][c] = m0; s.M[1][c] = m1; s.M[2][c] = m2; s.M[3][c] = m3;
  }
  const float e0 = q.t - m[3], e1 = q.d[0] - m[4], e2 = q.d[1] - m[5], e3 = q.d[2] - m[6];
  s.v[0] = e0 * d0;
  s.v[1] = (e1 - L[13] * s.v[0]) * d1;
  s.v[2] = (e2 - L[18] * s.v[0] - L[19] * s.v[1]) * d2;
  s.v[3] = (e3 - L[24] * s.v[0] - L[25] * s.v[1] - L[26] * s.v[2]) * d3;

  float G[3][3], u[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    u[a] = s.M[0][a] * s.v[0] + s.M[1][a] * s.v[1] + s.M[2][a] * s.v[2] + s.M[3][a] * s.v[3];
#pragma unroll
    for (int b = 0; b <= a; ++b) {
      G[a][b] = (a == b ? 1.f : 0.f) + s.M[0][a] * s.M[0][b] + s.M[1][a] * s.M[1][b] +
                s.M[2][a] * s.M[2][b] + s.M[3][a] * s.M[3][b];
    }
  }
  // H = chol(G)
  float (&H)[3][3] = s.H;
  H[0][0] = sqrtf(G[0][0]);
  const float ih0 = 1.f / H[0][0];
  H[1][0] = G[1][0] * ih0;
  H[2][0] = G[2][0] * ih0;
  H[1][1] = sqrtf(G[1][1] - H[1][0] * H[1][0]);
  const float ih1 = 1.f / H[1][1];
  H[2][1] = (G[2][1] - H[2][0] * H[1][0]) * ih1;
  H[2][2] = sqrtf(G[2][2] - H[2][0] * H[2][0] - H[2][1] * H[2][1]);
  const float ih2 = 1.f / H[2][2];
  H[0][1] = H[0][2] = H[1][2] = 0.f;
  s.z[0] = u[0] * ih0;
  s.z[1] = (u[1] - H[1][0] * s.z[0]) * ih1;
  s.z[2] = (u[2] - H[2][0] * s.z[0] - H[2][1] * s.z[1]) * ih2;
  // A = L11 H^-T, row by row: H a^T = l^T
  const float L11[3][3] = {{L[0], 0.f, 0.f}, {L[1], L[2], 0.f}, {L[3], L[4], L[5]}};
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const float a0 = L11[r][0] * ih0;
    const float a1 = (L11[r][1] - H[1][0] * a0) * ih1;
    const float a2 = (L11[r][2] - H[2][0] * a0 - H[2][1] * a1) * ih2;
    s.A[r][0] = a0; s.A[r][1] = a1; s.A[r][2] = a2;
  }
#pragma unroll
  for (int r = 0; r < 3; ++r)
    s.mu[r] = m[r] + s.A[r][0] * s.z[0] + s.A[r][1] * s.z[1] + s.A[r][2] * s.z[2];

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
  C[0][0] = sqrtf(S44);
  const float ic0 = 1.f / C[0][0];
  C[1][0] = S54 * ic0;
  C[2][0] = S64 * ic0;
  C[1][1] = sqrtf(S55 - C[1][0] * C[1][0]);
  const float ic1 = 1.f / C[1][1];
  C[2][1] = (S65 - C[2][0] * C[1][0]) * ic1;
  C[2][2] = sqrtf(S66 - C[2][0] * C[2][0] - C[2][1] * C[2][1]);
  const float ic2 = 1.f / C[2][2];
  C[0][1] = C[0][2] = C[1][2] = 0.f;
  s.y[0] = e1 * ic0;
  s.y[1] = (e2 - C[1][0] * s.y[0]) * ic1;
  s.y[2] = (e3 - C[2][0] * s.y[0] - C[2][1] * s.y[1]) * ic2;
  s.e_t = -0.5f * q.lambda_t * e0 * e0 / s.St;
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
  const float rz = 1.f / z;
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
