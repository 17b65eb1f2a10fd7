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

// The forward's shared-memory layout, arranged for 16-byte broadcast reads: unit u's first-layer
// row (7 weights, then its bias) is two float4; hidden unit j of MLP m has its output weights
// contiguous (rows padded to a multiple of 4).
struct AgrFwdWeights {
  float4 w1[kUnits][2];
  float4 w2p[kHidden];      // rows 0-2 (phi_p), padded
  float4 w2t[kHidden];      // row 3 (phi_t), padded
  float4 w2d[kHidden];      // rows 4-6 (phi_d), padded
  float4 w2l[kHidden][7];   // rows 7-34 (phi_l)
  float b2[kOut];
};

__device__ __forceinline__ void load_fwd_weights(AgrFwdWeights& F, AgrWeights& W, const sdgs_agr& a, float t) {
  load_weights(W, a, t);  // gamma folded into W.bias
  for (int u = threadIdx.x; u < kUnits; u += blockDim.x) {
    F.w1[u][0] = make_float4(W.w1x[u][0], W.w1x[u][1], W.w1x[u][2], W.w1x[u][3]);
    F.w1[u][1] = make_float4(W.w1x[u][4], W.w1x[u][5], W.w1x[u][6], W.bias[u]);
  }
  for (int j = threadIdx.x; j < kHidden; j += blockDim.x) {
    F.w2p[j] = make_float4(W.w2[0][j], W.w2[1][j], W.w2[2][j], 0.f);
    F.w2t[j] = make_float4(W.w2[3][j], 0.f, 0.f, 0.f);
    F.w2d[j] = make_float4(W.w2[4][j], W.w2[5][j], W.w2[6][j], 0.f);
#pragma unroll
    for (int q = 0; q < 7; ++q)
      F.w2l[j][q] = make_float4(W.w2[7 + 4 * q][j], W.w2[8 + 4 * q][j], W.w2[9 + 4 * q][j], W.w2[10 + 4 * q][j]);
  }
  for (int r = threadIdx.x; r < kOut; r += blockDim.x) F.b2[r] = W.b2[r];
  __syncthreads();
}

__device__ __forceinline__ float fwd_hidden(const AgrFwdWeights& F, int u, const float x[kX]) {
  const float4 a = F.w1[u][0], b = F.w1[u][1];
  float z = b.w;  // same order as hidden_pre: bias, then columns 0..6
  z += a.x * x[0]; z += a.y * x[1]; z += a.z * x[2]; z += a.w * x[3];
  z += b.x * x[4]; z += b.y * x[5]; z += b.z * x[6];
  return fmaxf(z, 0.f);
}

__device__ __forceinline__ void agr_refine_one(const AgrFwdWeights& F, const float* __restrict__ mean7,
                                               const float* __restrict__ L28, int64_t i,
                                               float* __restrict__ mean7_out, float* __restrict__ L28_out);

__global__ void __launch_bounds__(kAgrThreads) agr_refine_kernel(const float* __restrict__ mean7,
                                                                 const float* __restrict__ L28, int64_t n,
                                                                 sdgs_agr agr, float t,
                                                                 float* __restrict__ mean7_out,
                                                                 float* __restrict__ L28_out) {
  __shared__ AgrWeights W;
  __shared__ AgrFwdWeights F;
  load_fwd_weights(F, W, agr, t);  // once per block: the grid strides over the Gaussians
  for (int64_t i = (int64_t)blockIdx.x * kAgrThreads + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * kAgrThreads)
    agr_refine_one(F, mean7, L28, i, mean7_out, L28_out);
}

__device__ __forceinline__ void agr_refine_one(const AgrFwdWeights& F, const float* __restrict__ mean7,
                                               const float* __restrict__ L28, int64_t i,
                                               float* __restrict__ mean7_out, float* __restrict__ L28_out) {
  float x[kX];
#pragma unroll
  for (int c = 0; c < kX; ++c) x[c] = mean7[kX * i + c];
  float out[kOut];
#pragma unroll
  for (int r = 0; r < kOut; ++r) out[r] = F.b2[r];
#pragma unroll 4
  for (int j = 0; j < kHidden; ++j) {  // phi_p
    const float h = fwd_hidden(F, j, x);
    const float4 w = F.w2p[j];
    out[0] += w.x * h; out[1] += w.y * h; out[2] += w.z * h;
  }
#pragma unroll 4
  for (int j = 0; j < kHidden; ++j) {  // phi_t
    const float h = fwd_hidden(F, kHidden + j, x);
    out[3] += F.w2t[j].x * h;
  }
#pragma unroll 4
  for (int j = 0; j < kHidden; ++j) {  // phi_d
    const float h = fwd_hidden(F, 2 * kHidden + j, x);
    const float4 w = F.w2d[j];
    out[4] += w.x * h; out[5] += w.y * h; out[6] += w.z * h;
  }
#pragma unroll 2
  for (int j = 0; j < kHidden; ++j) {  // phi_l
    const float h = fwd_hidden(F, 3 * kHidden + j, x);
#pragma unroll
    for (int q = 0; q < 7; ++q) {
      const float4 w = F.w2l[j][q];
      out[7 + 4 * q] += w.x * h; out[8 + 4 * q] += w.y * h; out[9 + 4 * q] += w.z * h; out[10 + 4 * q] += w.w * h;
    }
  }
#pragma unroll
  for (int c = 0; c < kX; ++c) mean7_out[kX * i + c] = x[c] + out[c];
  const float4* Lin = reinterpret_cast<const float4*>(L28 + 28 * i);
  float4* Lout = reinterpret_cast<float4*>(L28_out + 28 * i);
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    float4 l = Lin[q];
    l.x += out[kX + 4 * q]; l.y += out[kX + 4 * q + 1]; l.z += out[kX + 4 * q + 2]; l.w += out[kX + 4 * q + 3];
    Lout[q] = l;
  }
}

// Weight-gradient sums owned by the block: O1 = per unit (7 x-columns, then db1), O2 = per output
// row (64 hidden columns, then db2).
constexpr int kO1 = kUnits * (kX + 1);
constexpr int kO2 = kOut * (kHidden + 1);
constexpr int kPartial = kO1 + kO2;
constexpr int kOutPad = 36;  // dout rows padded to whole float4

struct AgrBwdShared {
  AgrWeights W;
  alignas(16) float x[kAgrThreads][kX + 1];      // the tile's x, then 1 (live) for the bias column
  alignas(16) float dout[kAgrThreads][kOutPad];  // gradients w.r.t. the 35 residuals, then 0
  float h[kAgrThreads][kHidden + 1];             // this MLP's hidden activations and dz (odd
  float dz[kAgrThreads][kHidden + 1];            // stride: rows written per thread conflict-free)
};
static_assert(sizeof(float) * kAgrThreads * (kHidden + 1) >= sizeof(float) * kPartial,
              "the final combine stages one half's sums in h");

// Weight-gradient sums of thread (j, half): hidden unit j of every MLP over the Gaussians of one
// half of each tile, kept in registers across tiles.  w1[m][c]: dW1 row m * 64 + j (7 x-columns,
// then the bias); w2[r]: dW2 column j of output row r; b2: the bias of output row tid % 35 for the
// 70 threads that own one.
struct AgrSums {
  float w1[kMlps][kX + 1];
  float w2[kOut];
  float b2;
};

// Adds MLP M's terms of the half's 64 Gaussians: x and dout are read as broadcast float4, dz and
// h once per Gaussian.
template <int M>
__device__ __forceinline__ void agr_weight_sums(const AgrBwdShared& S, int j, int half, AgrSums& acc) {
  constexpr int rb = row_begin(M), re = row_end(M);
  constexpr int q0 = rb / 4, q1 = (re + 3) / 4;  // float4 chunks of dout covering the rows
  const int g0 = half * (kAgrThreads / 2);
#pragma unroll 4
  for (int g = g0; g < g0 + kAgrThreads / 2; ++g) {
    const float dzj = S.dz[g][j];
    const float4 xa = *reinterpret_cast<const float4*>(&S.x[g][0]);
    const float4 xb = *reinterpret_cast<const float4*>(&S.x[g][4]);
    float* a1 = acc.w1[M];
    a1[0] += dzj * xa.x; a1[1] += dzj * xa.y; a1[2] += dzj * xa.z; a1[3] += dzj * xa.w;
    a1[4] += dzj * xb.x; a1[5] += dzj * xb.y; a1[6] += dzj * xb.z; a1[7] += dzj * xb.w;
    const float hj = S.h[g][j];
#pragma unroll
    for (int q = q0; q < q1; ++q) {
      const float4 d = *reinterpret_cast<const float4*>(&S.dout[g][4 * q]);
      const float dv[4] = {d.x, d.y, d.z, d.w};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int r = 4 * q + e;
        if (r >= rb && r < re) acc.w2[r] += dv[e] * hj;
      }
    }
  }
}

__global__ void __launch_bounds__(kAgrThreads) agr_bwd_kernel(
    const float* __restrict__ mean7, int64_t n, sdgs_agr agr, float t, const float* __restrict__ dmean7_hat,
    const float* __restrict__ dL28_hat, float* __restrict__ dmean7, float* __restrict__ dL28,
    float* __restrict__ partial) {
  extern __shared__ float4 s_dyn[];  // AgrBwdShared (above the 48 KB static limit)
  AgrBwdShared& S = *reinterpret_cast<AgrBwdShared*>(s_dyn);
  AgrWeights& W = S.W;
  float (*s_x)[kX + 1] = S.x;
  float (*s_dout)[kOutPad] = S.dout;
  float (*s_h)[kHidden + 1] = S.h;
  float (*s_dz)[kHidden + 1] = S.dz;
  load_weights(W, agr, t);
  const int tid = threadIdx.x;
  const int hj = tid & (kHidden - 1), half = tid / kHidden;  // this thread's weight-gradient sums
  AgrSums acc;
#pragma unroll
  for (int m = 0; m < kMlps; ++m)
#pragma unroll
    for (int c = 0; c <= kX; ++c) acc.w1[m][c] = 0.f;
#pragma unroll
  for (int r = 0; r < kOut; ++r) acc.w2[r] = 0.f;
  acc.b2 = 0.f;

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
    s_dout[tid][kOut] = 0.f;
    __syncthreads();  // the tile's x and dout are in
    if (tid < 2 * kOut) {  // bias of output row tid % 35 over the half's Gaussians (dout is 0 past the end)
      const int r = tid % kOut, g0 = (tid / kOut) * (kAgrThreads / 2);
#pragma unroll 8
      for (int g = g0; g < g0 + kAgrThreads / 2; ++g) acc.b2 += s_dout[g][r];
    }
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
      // this MLP's weight-gradient terms of the tile's Gaussians
      if (m == 0) agr_weight_sums<0>(S, hj, half, acc);
      if (m == 1) agr_weight_sums<1>(S, hj, half, acc);
      if (m == 2) agr_weight_sums<2>(S, hj, half, acc);
      if (m == 3) agr_weight_sums<3>(S, hj, half, acc);
    }
    if (live) {
#pragma unroll
      for (int c = 0; c < kX; ++c) dmean7[kX * i + c] += dmean7_hat[kX * i + c] + dx[c];
      if (dL28 != nullptr) {  // (NULL: the caller takes dL28_hat as the gradient of L28 itself)
#pragma unroll
        for (int k = 0; k < 28; ++k) dL28[28 * i + k] += dL28_hat[28 * i + k];
      }
    }
    __syncthreads();  // s_x / s_dout are rewritten by the next tile
  }
  // the block's sums: the second half's staged in shared memory, added to the first half's
  float* stage = &S.h[0][0];
  float* mine = partial + (size_t)blockIdx.x * kPartial;
  __syncthreads();
  if (half == 1) {
#pragma unroll
    for (int m = 0; m < kMlps; ++m)
#pragma unroll
      for (int c = 0; c <= kX; ++c) stage[(m * kHidden + hj) * (kX + 1) + c] = acc.w1[m][c];
#pragma unroll
    for (int r = 0; r < kOut; ++r) stage[kO1 + r * (kHidden + 1) + hj] = acc.w2[r];
  }
  if (tid >= kOut && tid < 2 * kOut) stage[kO1 + (tid - kOut) * (kHidden + 1) + kHidden] = acc.b2;
  __syncthreads();
  if (half == 0) {
#pragma unroll
    for (int m = 0; m < kMlps; ++m)
#pragma unroll
      for (int c = 0; c <= kX; ++c) {
        const int o = (m * kHidden + hj) * (kX + 1) + c;
        mine[o] = acc.w1[m][c] + stage[o];
      }
#pragma unroll
    for (int r = 0; r < kOut; ++r) {
      const int o = kO1 + r * (kHidden + 1) + hj;
      mine[o] = acc.w2[r] + stage[o];
    }
  }
  if (tid < kOut) {
    const int o = kO1 + tid * (kHidden + 1) + kHidden;
    mine[o] = acc.b2 + stage[o];
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
  return (int)std::min<int64_t>(tiles, 2 * (int64_t)device_sm_count());
}

}  // namespace

size_t agr_bwd_workspace_bytes(int64_t n) { return sizeof(float) * (size_t)kPartial * std::max(1, agr_bwd_blocks(n)); }

cudaError_t launch_agr_refine(const sdgs_scene& s, const sdgs_agr& a, float t, float* mean7_out, float* L28_out,
                              cudaStream_t st) {
  if (s.n == 0) return cudaSuccess;
  const int64_t tiles = (s.n + kAgrThreads - 1) / kAgrThreads;
  agr_refine_kernel<<<(unsigned)std::min<int64_t>(tiles, 4 * (int64_t)device_sm_count()), kAgrThreads, 0, st>>>(
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
