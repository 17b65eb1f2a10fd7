// Densification statistics of the conditional 3D Gaussians (Algorithm 1 step 7, Sec. 4.4): scale
// and rotation of Sigma_cond, the space-time coupling |Sigma_pt|, the temporal scale sqrt(Sigma_t),
// and the split / prune decisions.  One thread per Gaussian.
#include "geometry.cuh"

namespace sdgs {

namespace {

struct DensifyArgs {
  const float* mean7;
  const float* L28;
  const float* opacity;
  int64_t n;
  Query q;
  sdgs_densify_cfg cfg;
  sdgs_densify out;
};

// Sigma_cond = A A^T with A the 3x3 factor slicing produces.  One-sided (Hestenes) Jacobi on the
// columns of M = A^T (the rows of A) accumulates V with A^T V = W diag(S), so A = V diag(S) W^T
// and Sigma_cond = V diag(S)^2 V^T: S are the singular values of A (accurate even for very flat
// Gaussians, unlike eigenvalues of the product) and V the rotation.
__device__ __forceinline__ void scale_rotation(const float A[3][3], float S[3], float R[3][3]) {
  float m[3][3], v[3][3];
#pragma unroll
  for (int j = 0; j < 3; ++j)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      m[j][k] = A[j][k];
      v[k][j] = j == k ? 1.f : 0.f;  // v[row][col]; column j pairs with m[j]
    }
#pragma unroll 1
  for (int sweep = 0; sweep < 8; ++sweep) {
#pragma unroll
    for (int pq = 0; pq < 3; ++pq) {
      const int p = pq == 2 ? 1 : 0, q = pq == 0 ? 1 : 2;
      const float al = m[p][0] * m[p][0] + m[p][1] * m[p][1] + m[p][2] * m[p][2];
      const float be = m[q][0] * m[q][0] + m[q][1] * m[q][1] + m[q][2] * m[q][2];
      const float ga = m[p][0] * m[q][0] + m[p][1] * m[q][1] + m[p][2] * m[q][2];
      if (!(fabsf(ga) > 1e-30f) || !(fabsf(ga) > 1e-9f * sqrtf(al * be))) continue;
      const float zeta = (be - al) / (2.f * ga);
      const float t = copysignf(1.f, zeta) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
      const float c = 1.f / sqrtf(1.f + t * t), s = c * t;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float mp = m[p][k], mq = m[q][k];
        m[p][k] = c * mp - s * mq;
        m[q][k] = s * mp + c * mq;
        const float vp = v[k][p], vq = v[k][q];
        v[k][p] = c * vp - s * vq;
        v[k][q] = s * vp + c * vq;
      }
    }
  }
  float sv[3];
  int idx[3] = {0, 1, 2};
#pragma unroll
  for (int j = 0; j < 3; ++j) sv[j] = sqrtf(m[j][0] * m[j][0] + m[j][1] * m[j][1] + m[j][2] * m[j][2]);
  // descending order (3-element sorting network on indices)
  auto cswap = [&](int a, int b) {
    if (sv[idx[a]] < sv[idx[b]]) { const int t = idx[a]; idx[a] = idx[b]; idx[b] = t; }
  };
  cswap(0, 1); cswap(1, 2); cswap(0, 1);
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    S[j] = sv[idx[j]];
#pragma unroll
    for (int r = 0; r < 3; ++r) R[r][j] = v[r][idx[j]];
  }
  // a proper rotation: last column times sign(det R)
  const float det = R[0][0] * (R[1][1] * R[2][2] - R[1][2] * R[2][1]) -
                    R[0][1] * (R[1][0] * R[2][2] - R[1][2] * R[2][0]) +
                    R[0][2] * (R[1][0] * R[2][1] - R[1][1] * R[2][0]);
  if (det < 0.f) {
#pragma unroll
    for (int r = 0; r < 3; ++r) R[r][2] = -R[r][2];
  }
}

__global__ void __launch_bounds__(128) densify_kernel(const DensifyArgs a) {
  const int64_t i = (int64_t)blockIdx.x * 128 + threadIdx.x;
  if (i >= a.n) return;
  float L[28];
  const float4* Lp = reinterpret_cast<const float4*>(a.L28 + 28 * i);
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    const float4 w = __ldg(Lp + k);
    L[4 * k] = w.x; L[4 * k + 1] = w.y; L[4 * k + 2] = w.z; L[4 * k + 3] = w.w;
  }
  float m[7];
#pragma unroll
  for (int k = 0; k < 7; ++k) m[k] = __ldg(a.mean7 + 7 * i + k);
  const float alpha = __ldg(a.opacity + i);
  float rnd;
  const Query q = query_for(a.q, m, &rnd);
  SliceState s;
  slice_one(L, m, alpha, q, s);
  const sdgs_densify& o = a.out;
  if (o.scale || o.rot) {
    float S[3], R[3][3];
    scale_rotation(s.A, S, R);
    if (o.scale)
#pragma unroll
      for (int j = 0; j < 3; ++j) o.scale[3 * i + j] = S[j];
    if (o.rot)
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) o.rot[9 * i + 3 * r + c] = R[r][c];
  }
  // Sigma_pt[r] = (row r of L) . (row 3 of L); Sigma_t = |row 3 of L|^2
  const float* lt = L + 6;
  const float pt0 = L[0] * lt[0];
  const float pt1 = L[1] * lt[0] + L[2] * lt[1];
  const float pt2 = L[3] * lt[0] + L[4] * lt[1] + L[5] * lt[2];
  const float pt_norm = sqrtf(pt0 * pt0 + pt1 * pt1 + pt2 * pt2);
  const float t_scale = sqrtf(s.St);
  if (o.pt_norm) o.pt_norm[i] = pt_norm;
  if (o.t_scale) o.t_scale[i] = t_scale;
  if (o.split) o.split[i] = (pt_norm > a.cfg.split_pt * a.cfg.extent) && (t_scale > a.cfg.split_t);
  if (o.prune) o.prune[i] = alpha < a.cfg.prune_alpha;
}

}  // namespace

cudaError_t launch_densify(const sdgs_scene& s, const sdgs_view& v, const sdgs_densify_cfg& cfg,
                           const sdgs_densify& out, cudaStream_t st) {
  if (s.n == 0) return cudaSuccess;
  DensifyArgs a;
  a.mean7 = s.mean7; a.L28 = s.L28; a.opacity = s.opacity; a.n = s.n;
  a.q = make_query(s, v);
  a.cfg = cfg;
  a.out = out;
  densify_kernel<<<(unsigned)((s.n + 127) / 128), 128, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace sdgs
