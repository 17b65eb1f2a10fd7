// Adaptive Gaussian Refinement (Sec. 4.3, Algorithm 1 steps 1-2): four MLPs 27 -> 64 -> {3, 1, 3, 28}
// on f = mu_p (+) mu_t (+) mu_d (+) gamma(t) add residuals to the 7D means and the packed L.
//
// Layer 1 splits into a per-request part -- the 20 columns that read gamma(t), folded with b1 into
// one bias per hidden unit -- and a per-Gaussian 7-column part.  Weights live in shared memory and
// every thread refines one Gaussian in FP32 (the contraction per Gaussian is 256 x 7 + 35 x 64
// multiply-adds, too narrow and too precision-sensitive for the tensor cores to pay).  The backward
// recomputes the hidden layer, forms the input gradient per Gaussian and accumulates the weight
// gradients per block over tiles of Gaussians (block-level sums in shared memory, one partial per
// block), reduced across blocks in a fixed order.
#include <math.h>

#include <algorithm>

#include "common.cuh"

namespace sdgs {

namespace {

constexpr int kIn = 27, kX = 7, kHidden = 64, kMlps = 4, kUnits = kMlps * kHidden, kOut = 35;
constexpr int kFreq = 10;
constexpr int kAgrThreads = 128;
__host__ __device__ constexpr int row_begin(int m) { return m == 0 ? 0 : m == 1 ? 3 : m == 2 ? 4 : 7; }
__host__ __device__ constexpr int row_end(int m) { return m == 0 ? 3 : m == 1 ? 4 : m == 2 ? 7 : 35; }

struct AgrWeights {  // shared-memory copy with the per-request bias folded in
  float w1x[kUnits][kX];
  float bias[kUnits];  // b1 + w1[:, 7:27] gamma(t)
  float w2[kOut][kHidden];
  float b2[kOut];
  float gamma[2 * kFreq];
};

// gamma(t): sin(2^k pi t), cos(2^k pi t); 2^k t is exact in FP32, so sinpif / cospif see the exact
// argument.
__device__ __forceinline__ void load_weights(AgrWeights& W, const sdgs_agr& a, float t) {
  for (int k = threadIdx.x; k < kFreq; k += blockDim.x) {
    const float x = ldexpf(t, k);
    W.gamma[2 * k] = sinpif(x);
    W.gamma[2 * k + 1] = cospif(x);
  }
  for (int i = threadIdx.x; i < kOut * kHidden; i += blockDim.x) (&W.w2[0][0])[i] = a.w2[i];
  for (int i = threadIdx.x; i < kOut; i += blockDim.x) W.b2[i] = a.b2[i];
  for (int i = threadIdx.x; i < kUnits * kX; i += blockDim.x) W.w1x[i / kX][i % kX] = a.w1[(i / kX) * kIn + i % kX];
  __syncthreads();
  for (int u = threadIdx.x; u < kUnits; u += blockDim.x) {
    float b = a.b1[u];
    const float* w = a.w1 + u * kIn + kX;
#pragma unroll
    for (int c = 0; c < 2 * kFreq; ++c) b += w[c] * W.gamma[c];
    W.bias[u] = b;
  }
  __syncthreads();
}

__device__ __forceinline__ float hidden_pre(const AgrWeights& W, int u, const float x[kX]) {
  float z = W.bias[u];
#pragma unroll
  for (int c = 0; c < kX; ++c) z += W.w1x[u][c] * x[c];
  return z;
}

__global__ void __launch_bounds__(kAgrThreads) agr_refine_kernel(const float* __restrict__ mean7,
                                                                 const float* __restrict__ L28, int64_t n,
                                                                 sdgs_agr agr, float t,
                                                                 float* __restrict__ mean7_out,
                                                                 float* __restrict__ L28_out) {
  __shared__ AgrWeights W;
  load_weights(W, agr, t);
  const int64_t i = (int64_t)blockIdx.x * kAgrThreads + threadIdx.x;
  if (i >= n) return;
  float x[kX];
#pragma unroll
  for (int c = 0; c < kX; ++c) x[c] = mean7[kX * i + c];
  float out[kOut];
#pragma unroll
  for (int r = 0; r < kOut; ++r) out[r] = W.b2[r];
#pragma unroll
  for (int m = 0; m < kMlps; ++m) {
#pragma unroll 4
    for (int j = 0; j < kHidden; ++j) {
      const float h = fmaxf(hidden_pre(W, m * kHidden + j, x), 0.f);
#pragma unroll
      for (int r = row_begin(m); r < row_end(m); ++r) out[r] += W.w2[r][j] * h;
    }
  }
#pragma unroll
  for (int c = 0; c < kX; ++c) mean7_out[kX * i + c] = x[c] + out[c];
#pragma unroll
  for (int k = 0; k < 28; ++k) L28_out[28 * i + k] = L28[28 * i + k] + out[kX + k];
}

// Weight-gradient sums owned by the block: O1 = per unit (7 x-columns, then db1), O2 = per output
// row (64 hidden columns, then db2).
constexpr int kO1 = kUnits * (kX + 1);
constexpr int kO2 = kOut * (kHidden + 1);
constexpr int kPartial = kO1 + kO2;
constexpr int kAcc1 = kO1 / kAgrThreads;                          // 16 per thread
constexpr int kAcc2 = (kO2 + kAgrThreads - 1) / kAgrThreads;      // 18 per thread

struct AgrBwdShared {
  AgrWeights W;
  float x[kAgrThreads][kX + 1];      // the tile's x, then 1 (live) for the bias column
  float dout[kAgrThreads][kOut];     // gradients w.r.t. the 35 residuals
  float h[kAgrThreads][kHidden + 1]; // this MLP's hidden activations, then 1 (live)
  float dz[kAgrThreads][kHidden + 1];
};

__global__ void __launch_bounds__(kAgrThreads) agr_bwd_kernel(
    const float* __restrict__ mean7, int64_t n, sdgs_agr agr, float t, const float* __restrict__ dmean7_hat,
    const float* __restrict__ dL28_hat, float* __restrict__ dmean7, float* __restrict__ dL28,
    float* __restrict__ partial) {
  extern __shared__ float4 s_dyn[];  // AgrBwdShared (above the 48 KB static limit)
  AgrBwdShared& S = *reinterpret_cast<AgrBwdShared*>(s_dyn);
  AgrWeights& W = S.W;
  float (*s_x)[kX + 1] = S.x;
  float (*s_dout)[kOut] = S.dout;
  float (*s_h)[kHidden + 1] = S.h;
  float (*s_dz)[kHidden + 1] = S.dz;
  load_weights(W, agr, t);
  const int tid = threadIdx.x;
  float acc1[kAcc1], acc2[kAcc2];
#pragma unroll
  for (int k = 0; k < kAcc1; ++k) acc1[k] = 0.f;
#pragma unroll
  for (int k = 0; k < kAcc2; ++k) acc2[k] = 0.f;

  const int64_t tiles = (n + kAgrThreads - 1) / kAgrThreads;
  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int64_t i = tile * kAgrThreads + tid;
    const bool live = i < n;
    float x[kX], dout[kOut], dx[kX];
#pragma unroll
    for (int c = 0; c < kX; ++c) {
      x[c] = live ? mean7[kX * i + c] : 0.f;
      dx[c] = 0.f;
      s_x[tid][c] = x[c];
    }
    s_x[tid][kX] = live ? 1.f : 0.f;
#pragma unroll
    for (int r = 0; r < kX; ++r) dout[r] = live ? dmean7_hat[kX * i + r] : 0.f;
#pragma unroll
    for (int r = kX; r < kOut; ++r) dout[r] = live ? dL28_hat[28 * i + r - kX] : 0.f;
#pragma unroll
    for (int r = 0; r < kOut; ++r) s_dout[tid][r] = dout[r];
#pragma unroll
    for (int m = 0; m < kMlps; ++m) {
      __syncthreads();  // the previous MLP's sums are done with s_h / s_dz
#pragma unroll 2
      for (int j = 0; j < kHidden; ++j) {
        const int u = m * kHidden + j;
        const float z = hidden_pre(W, u, x);
        float dh = 0.f;
#pragma unroll
        for (int r = row_begin(m); r < row_end(m); ++r) dh += W.w2[r][j] * dout[r];
        const float dz = z > 0.f ? dh : 0.f;
        s_h[tid][j] = fmaxf(z, 0.f);
        s_dz[tid][j] = dz;
#pragma unroll
        for (int c = 0; c < kX; ++c) dx[c] += W.w1x[u][c] * dz;
      }
      s_h[tid][kHidden] = live ? 1.f : 0.f;
      __syncthreads();
      // this MLP's weight-gradient sums over the tile's Gaussians
#pragma unroll
      for (int k = 0; k < kAcc1; ++k) {
        const int o = tid + k * kAgrThreads;
        if (o / ((kX + 1) * kHidden) != m) continue;
        const int j = (o / (kX + 1)) % kHidden, c = o % (kX + 1);
        float s = 0.f;
#pragma unroll 8
        for (int g = 0; g < kAgrThreads; ++g) s += s_dz[g][j] * s_x[g][c];
        acc1[k] += s;
      }
#pragma unroll
      for (int k = 0; k < kAcc2; ++k) {
        const int o = tid + k * kAgrThreads;
        if (o >= kO2) continue;
        const int r = o / (kHidden + 1), j = o % (kHidden + 1);
        if (r < row_begin(m) || r >= row_end(m)) continue;
        float s = 0.f;
#pragma unroll 8
        for (int g = 0; g < kAgrThreads; ++g) s += s_dout[g][r] * s_h[g][j];
        acc2[k] += s;
      }
    }
    if (live) {
#pragma unroll
      for (int c = 0; c < kX; ++c) dmean7[kX * i + c] += dmean7_hat[kX * i + c] + dx[c];
#pragma unroll
      for (int k = 0; k < 28; ++k) dL28[28 * i + k] += dL28_hat[28 * i + k];
    }
    __syncthreads();  // s_x / s_dout are rewritten by the next tile
  }
  float* mine = partial + (size_t)blockIdx.x * kPartial;
#pragma unroll
  for (int k = 0; k < kAcc1; ++k) mine[tid + k * kAgrThreads] = acc1[k];
#pragma unroll
  for (int k = 0; k < kAcc2; ++k) {
    const int o = tid + k * kAgrThreads;
    if (o < kO2) mine[kO1 + o] = acc2[k];
  }
}

// Sums the blocks' partials in block order and adds them to the caller's weight gradients; the
// 20 gamma columns of w1 get gamma[c] times the unit's bias gradient.
__global__ void agr_reduce_kernel(const float* __restrict__ partial, int blocks, float t, sdgs_agr_grads g) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= kPartial) return;
  float s = 0.f;
  for (int b = 0; b < blocks; ++b) s += partial[(size_t)b * kPartial + o];
  if (o < kO1) {
    const int u = o / (kX + 1), c = o % (kX + 1);
    if (c < kX) {
      g.dw1[u * kIn + c] += s;
    } else {
      g.db1[u] += s;
      for (int k = 0; k < kFreq; ++k) {
        const float x = ldexpf(t, k);
        g.dw1[u * kIn + kX + 2 * k] += s * sinpif(x);
        g.dw1[u * kIn + kX + 2 * k + 1] += s * cospif(x);
      }
    }
  } else {
    const int q = o - kO1, r = q / (kHidden + 1), j = q % (kHidden + 1);
    if (j < kHidden) g.dw2[r * kHidden + j] += s;
    else g.db2[r] += s;
  }
}

int agr_bwd_blocks(int64_t n) {
  const int64_t tiles = (n + kAgrThreads - 1) / kAgrThreads;
  return (int)std::min<int64_t>(tiles, 2 * 152);
}

}  // namespace

size_t agr_bwd_workspace_bytes(int64_t n) { return sizeof(float) * (size_t)kPartial * std::max(1, agr_bwd_blocks(n)); }

cudaError_t launch_agr_refine(const sdgs_scene& s, const sdgs_agr& a, float t, float* mean7_out, float* L28_out,
                              cudaStream_t st) {
  if (s.n == 0) return cudaSuccess;
  agr_refine_kernel<<<(unsigned)((s.n + kAgrThreads - 1) / kAgrThreads), kAgrThreads, 0, st>>>(
      s.mean7, s.L28, s.n, a, t, mean7_out, L28_out);
  return cudaGetLastError();
}

cudaError_t launch_agr_refine_bwd(const sdgs_scene& s, const sdgs_agr& a, float t, const float* dmean7_hat,
                                  const float* dL28_hat, float* dmean7, float* dL28, const sdgs_agr_grads& g,
                                  char* ws, cudaStream_t st) {
  if (s.n == 0) return cudaSuccess;
  const int blocks = agr_bwd_blocks(s.n);
  float* partial = reinterpret_cast<float*>(ws);
  cudaError_t e = cudaFuncSetAttribute(agr_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sizeof(AgrBwdShared));  // for the current device
  if (e != cudaSuccess) return e;
  agr_bwd_kernel<<<blocks, kAgrThreads, sizeof(AgrBwdShared), st>>>(s.mean7, s.n, a, t, dmean7_hat, dL28_hat,
                                                                     dmean7, dL28, partial);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  agr_reduce_kernel<<<(kPartial + 255) / 256, 256, 0, st>>>(partial, blocks, t, g);
  return cudaGetLastError();
}

}  // namespace sdgs
