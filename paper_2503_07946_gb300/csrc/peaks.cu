// Throughput probes of the SM pipes the rasteriser is bound by: scalar FP32 FMA, paired FP32 FMA
// (two lanes' worth per instruction) and the MUFU ex2.  Each thread runs kChains independent
// dependency chains so that issue, not latency, limits the rate; the chains' results go to `sink`
// so that nothing is optimised away.  The caller times a launch and divides the operation count by
// the time: the measured peaks of this GPU at the clock it ran at.
#include "common.cuh"
#include "raster_common.cuh"

namespace sdgs {

namespace {

constexpr int kProbeThreads = 256;
constexpr int kChains = 8;

__global__ void __launch_bounds__(kProbeThreads) ffma_probe_kernel(int iters, float a, float b, float* sink) {
  float x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (float)(threadIdx.x + c) * 1e-3f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = __fmaf_rn(x[c], a, b);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  sink[(size_t)blockIdx.x * kProbeThreads + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kProbeThreads) ffma2_probe_kernel(int iters, float a, float b, float* sink) {
  float2 x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = make_float2((float)(threadIdx.x + c) * 1e-3f, (float)c * 1e-3f);
  const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = __ffma2_rn(x[c], a2, b2);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c].x + x[c].y;
  sink[(size_t)blockIdx.x * kProbeThreads + threadIdx.x] = s;
}

// y <- 2^(-y) keeps every chain in (0.5, 1).
__global__ void __launch_bounds__(kProbeThreads) ex2_probe_kernel(int iters, float* sink) {
  float y[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) y[c] = 0.5f + (float)((threadIdx.x + c) & 63) * (0.5f / 64.f);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) y[c] = ex2_approx(-y[c]);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += y[c];
  sink[(size_t)blockIdx.x * kProbeThreads + threadIdx.x] = s;
}

}  // namespace

int64_t alu_probe_sink_len() { return (int64_t)device_sm_count() * 8 * kProbeThreads; }

cudaError_t launch_alu_probe(int kind, int iters, float* sink, double* ops, cudaStream_t st) {
  const int blocks = device_sm_count() * 8;  // 64 warps per SM
  const double per_thread = (double)iters * 4 * kChains;
  const double threads = (double)blocks * kProbeThreads;
  switch (kind) {
    case 0:
      ffma_probe_kernel<<<blocks, kProbeThreads, 0, st>>>(iters, 0.999f, 1e-3f, sink);
      *ops = 2.0 * per_thread * threads;  // FLOP: an FMA is 2
      break;
    case 1:
      ffma2_probe_kernel<<<blocks, kProbeThreads, 0, st>>>(iters, 0.999f, 1e-3f, sink);
      *ops = 4.0 * per_thread * threads;  // two FMAs per instruction
      break;
    default:
      ex2_probe_kernel<<<blocks, kProbeThreads, 0, st>>>(iters, sink);
      *ops = per_thread * threads;  // ex2 evaluations
      break;
  }
  return cudaGetLastError();
}

}  // namespace sdgs
