// Shared device helpers for the agent-based image solver kernels (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace agents {

constexpr int kWarp = 32;

// C2 Wendland kernel of Eq. kernel, read as phi(r) = (1 - r)^4 (4 r + 1) on [0, 1] and
// 0 beyond, with its derivative phi'(r) = -20 r (1 - r)^3.  Clamping r at 1 makes both
// vanish exactly past the support without a branch (t = 0 there).
__device__ __forceinline__ float wendland_phi(float r) {
  const float rc = fminf(r, 1.0f);
  const float t = 1.0f - rc;
  const float t2 = t * t;
  return (t2 * t2) * fmaf(4.0f, rc, 1.0f);
}

__device__ __forceinline__ void wendland_phi_dphi(float r, float& phi, float& dphi) {
  const float rc = fminf(r, 1.0f);
  const float t = 1.0f - rc;
  const float t2 = t * t;
  phi = (t2 * t2) * fmaf(4.0f, rc, 1.0f);
  dphi = (-20.0f * rc) * (t2 * t);
}

// The same functions of s = 1 - r, for callers that form 1 - r directly with one FMA:
// with t = max(s, 0), phi = t^4 (5 - 4t) and phi' = 20 t^3 (t - 1) (both 0 for r >= 1).
__device__ __forceinline__ float wendland_phi_1m(float s) {
  const float t = fmaxf(s, 0.0f);
  const float t2 = t * t;
  return (t2 * t2) * fmaf(-4.0f, t, 5.0f);
}

__device__ __forceinline__ void wendland_phi_dphi_1m(float s, float& phi, float& dphi) {
  const float t = fmaxf(s, 0.0f);
  const float t2 = t * t;
  const float t3 = t2 * t;
  phi = (t2 * t2) * fmaf(-4.0f, t, 5.0f);
  dphi = (20.0f * t3) * (t - 1.0f);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int off = kWarp / 2; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  return v;
}

// Deterministic block sum of NV doubles per thread: fixed shuffle tree inside each warp,
// then warp 0 adds the per-warp results in warp order.  `red` must hold NV * nwarps
// doubles.  Thread 0 receives the totals in out[] (other threads: unspecified).
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* red, double (&out)[NV]) {
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int nthreads = blockDim.x * blockDim.y * blockDim.z;
  const int nwarps = (nthreads + kWarp - 1) / kWarp;
  const int lane = tid & (kWarp - 1), warp = tid / kWarp;
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) red[k * nwarps + warp] = v[k];
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double s = lane < nwarps ? red[k * nwarps + lane] : 0.0;
      s = warp_sum(s);
      if (lane == 0) out[k] = s;
    }
  }
}

}  // namespace agents
