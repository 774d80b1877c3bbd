// FP32 throughput probe for the roofline of the agent sweeps, which are bound by the
// FP32 pipe: independent FMA chains per thread, no memory traffic, a full grid.  The
// benchmark times one launch with CUDA events and divides the flop count this file
// reports by it; that measured rate is the denominator of the sweeps' roofline fraction.
//
// Two forms: scalar FFMA (16 independent chains per thread) and packed FFMA2 on float2
// (8 chains of two lanes, the form the sweep kernels issue).  Each chain is
// x <- x * a + b with |a| < 1, so values stay finite and normal; a and b are kernel
// arguments, so nothing folds at compile time.  The result is stored only if it equals a
// value it never takes (the compiler cannot prove that), which keeps every chain live.
#include "agents.h"

#include <cuda_runtime.h>

namespace {

constexpr int kThreads = 256;
constexpr int kChains = 16;   // FMAs per thread and iteration, both forms

__global__ void __launch_bounds__(kThreads) fma_probe_scalar(float* sink, int iters, float a,
                                                            float b) {
  float x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = (float)(threadIdx.x + k) * 1e-3f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = fmaf(x[k], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  if (s == -1.0f) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) fma_probe_packed(float* sink, int iters, float a,
                                                            float b) {
  float2 x[kChains / 2];
#pragma unroll
  for (int k = 0; k < kChains / 2; ++k)
    x[k] = make_float2((float)(threadIdx.x + k) * 1e-3f, (float)(threadIdx.x - k) * 1e-3f);
  const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains / 2; ++k) x[k] = __ffma2_rn(x[k], a2, b2);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains / 2; ++k) s += x[k].x + x[k].y;
  if (s == -1.0f) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" int agents_fp32_probe(int32_t packed, int32_t blocks, int32_t iters, float* sink_dev,
                                 void* cuda_stream, double* flops_out) {
  if (blocks < 1 || iters < 1 || !sink_dev || !flops_out) return AGENTS_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  if (packed)
    fma_probe_packed<<<blocks, kThreads, 0, s>>>(sink_dev, iters, 0.99999994f, 1e-7f);
  else
    fma_probe_scalar<<<blocks, kThreads, 0, s>>>(sink_dev, iters, 0.99999994f, 1e-7f);
  if (cudaGetLastError() != cudaSuccess) return AGENTS_ECUDA;
  *flops_out = 2.0 * kChains * (double)kThreads * (double)blocks * (double)iters;
  return AGENTS_OK;
}
