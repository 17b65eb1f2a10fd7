// Forward per-Gaussian kernel: conditional slicing + modulation + cull + EWA projection + SH
// colour, fused into one pass over the scene (one thread per Gaussian).
#include <string.h>

#include <algorithm>

#include "geometry.cuh"

namespace sdgs {

namespace {

struct SliceArgs {
  const float* mean7;
  const float* L28;
  const float* opacity;
  const float* sh;
  int64_t n;
  Query q;
  Camera cam;
  float2* mean2d;
  float4* conic_opacity;
  float* rgb;
  float* depth;
  ushort4* rect;
  int32_t* radius;
};

constexpr int kThreads = 128;

// One launch slices up to kMaxSliceBatch problems (blockIdx.y selects one), their arguments by
// value in kernel parameter space; a single problem is a batch of one, so a request sliced in a
// batch gives the same bits as the request sliced alone.
constexpr int kMaxSliceBatch = kMaxBinBatch;
struct SliceBatch {
  SliceArgs a[kMaxSliceBatch];
};

__device__ __forceinline__ void slice_project_one(const SliceArgs& a, int64_t i);

__global__ void __launch_bounds__(kThreads) slice_project_kernel(const SliceBatch b) {
  griddep_wait();
  const SliceArgs& a = b.a[blockIdx.y];
  const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (i >= a.n) return;
  slice_project_one(a, i);
}

__device__ __forceinline__ void slice_project_one(const SliceArgs& a, int64_t i) {
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
  const float alpha = __ldg(a.opacity + i);

  SliceState s;
  float rnd;
  const Query qi = query_for(a.q, m, &rnd);
  const float alpha_c = slice_one(L, m, alpha, qi, s);
  ProjState ps;
  bool keep = alpha_c >= kAlphaMin && project_one(a.cam, s, ps);
  float u = 0.f, v = 0.f, r = 0.f;
  int rx0 = 0, ry0 = 0, rx1 = 0, ry1 = 0;
  if (keep) {
    const float rz = __fdividef(1.f, ps.p[2]);
    u = a.cam.fx * ps.p[0] * rz + a.cam.cx;
    v = a.cam.fy * ps.p[1] * rz + a.cam.cy;
    const float mid = 0.5f * (ps.cov[0] + ps.cov[2]);
    const float lam = mid + sqrtf(fmaxf(0.f, mid * mid - ps.det));
    r = ceilf(kExtent * sqrtf(lam));
    const float inv = 1.0f / kTile;
    rx0 = (int)fminf((float)a.cam.tiles_x, fmaxf(0.f, floorf((u - r) * inv)));
    rx1 = (int)fminf((float)a.cam.tiles_x, fmaxf(0.f, floorf((u + r) * inv) + 1.f));
    ry0 = (int)fminf((float)a.cam.tiles_y, fmaxf(0.f, floorf((v - r) * inv)));
    ry1 = (int)fminf((float)a.cam.tiles_y, fmaxf(0.f, floorf((v + r) * inv) + 1.f));
    keep = rx1 > rx0 && ry1 > ry0 && isfinite(r);
  }
  if (!keep) {
    a.rect[i] = make_ushort4(0, 0, 0, 0);
    a.radius[i] = 0;
    return;
  }
  const float idet = __fdividef(1.f, ps.det);
  a.mean2d[i] = make_float2(u, v);
  a.conic_opacity[i] = make_float4(ps.cov[2] * idet, -ps.cov[1] * idet, ps.cov[0] * idet, alpha_c);
  a.depth[i] = ps.p[2];
  a.rect[i] = make_ushort4((unsigned short)rx0, (unsigned short)ry0, (unsigned short)rx1,
                           (unsigned short)ry1);
  a.radius[i] = (int32_t)r;

  // SH colour toward the Gaussian from the camera centre.
  float dx = s.mu[0] - a.cam.campos[0], dy = s.mu[1] - a.cam.campos[1], dz = s.mu[2] - a.cam.campos[2];
  const float rn = rsqrtf(dx * dx + dy * dy + dz * dz);
  dx *= rn; dy *= rn; dz *= rn;
  float Y[16];
  sh_basis(dx, dy, dz, Y);
  const float4* shp = reinterpret_cast<const float4*>(a.sh + 48 * i);  // 192-byte rows: aligned
  float c[3] = {0.5f, 0.5f, 0.5f};
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    const float4 w = __ldg(shp + k);
    const float vals[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int flat = 4 * k + j;  // coefficient flat / 3, channel flat % 3
      c[flat % 3] += Y[flat / 3] * vals[j];
    }
  }
  a.rgb[3 * i + 0] = fmaxf(c[0], 0.f);
  a.rgb[3 * i + 1] = fmaxf(c[1], 0.f);
  a.rgb[3 * i + 2] = fmaxf(c[2], 0.f);
}

}  // namespace

Camera make_camera(const sdgs_view& v) {
  Camera c;
  for (int r = 0; r < 3; ++r) {
    for (int k = 0; k < 3; ++k) c.R[r][k] = v.viewmat[4 * r + k];
    c.T[r] = v.viewmat[4 * r + 3];
  }
  // camera centre = -R^T T
  for (int k = 0; k < 3; ++k)
    c.campos[k] = -(c.R[0][k] * c.T[0] + c.R[1][k] * c.T[1] + c.R[2][k] * c.T[2]);
  c.fx = v.fx; c.fy = v.fy; c.cx = v.cx; c.cy = v.cy;
  c.lim_x = kJacClamp * (0.5f * (float)v.width / v.fx);
  c.lim_y = kJacClamp * (0.5f * (float)v.height / v.fy);
  c.near_plane = v.near_plane;
  c.width = v.width; c.height = v.height;
  c.tiles_x = tiles_of(v.width);
  c.tiles_y = tiles_of(v.height);
  return c;
}

Query make_query(const sdgs_scene& s, const sdgs_view& v) {
  Query q;
  q.t = v.t;
  q.d[0] = v.d[0]; q.d[1] = v.d[1]; q.d[2] = v.d[2];
  q.lambda_t = s.lambda_t;
  q.lambda_d = s.lambda_d;
  q.dir_mode = s.dir_mode;
  const Camera c = make_camera(v);
  q.campos[0] = c.campos[0]; q.campos[1] = c.campos[1]; q.campos[2] = c.campos[2];
  return q;
}

static SliceArgs make_args(const sdgs_scene& s, const sdgs_view& v, const sdgs_projected& o);

cudaError_t launch_slice_project(const sdgs_scene& s, const sdgs_view& v, const sdgs_projected& o,
                                 cudaStream_t st) {
  const SliceRequest r{s, v, o};
  return launch_slice_project_batch(&r, 1, st);
}

cudaError_t launch_slice_project_batch(const SliceRequest* reqs, int count, cudaStream_t st) {
  for (int j0 = 0; j0 < count; j0 += kMaxSliceBatch) {
    SliceBatch b;
    int m = 0;
    int64_t max_n = 0;
    for (int j = j0; j < count && m < kMaxSliceBatch; ++j, ++m) {
      b.a[m] = make_args(reqs[j].scene, reqs[j].view, reqs[j].out);
      max_n = std::max<int64_t>(max_n, reqs[j].scene.n);
    }
    for (int k = m; k < kMaxSliceBatch; ++k) b.a[k] = b.a[0];  // (never read: grid.y = m)
    if (max_n == 0) continue;
    const int64_t blocks = (max_n + kThreads - 1) / kThreads;
    const cudaError_t e = launch_pdl(slice_project_kernel, dim3((unsigned)blocks, (unsigned)m), dim3(kThreads), 0, st, b);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

static SliceArgs make_args(const sdgs_scene& s, const sdgs_view& v, const sdgs_projected& o) {
  SliceArgs a;
  a.mean7 = s.mean7; a.L28 = s.L28; a.opacity = s.opacity; a.sh = s.sh; a.n = s.n;
  a.q = make_query(s, v);
  a.cam = make_camera(v);
  a.mean2d = reinterpret_cast<float2*>(o.mean2d);
  a.conic_opacity = reinterpret_cast<float4*>(o.conic_opacity);
  a.rgb = o.rgb;
  a.depth = o.depth;
  a.rect = reinterpret_cast<ushort4*>(o.rect);
  a.radius = o.radius;
  return a;
}

}  // namespace sdgs
