// Conversions between float32 and float64 done with integer operations on the IEEE 754
// bit patterns (binary32: 1 sign, 8 exponent bits with bias 127, 23 fraction bits;
// binary64: 1, 11 with bias 1023, 52).  On GB300 the hardware conversions execute on the
// float64 pipe, which the multiplier update saturates; these run on the integer units.
//  * widen: exact; a normal binary32 keeps its sign, re-biases its exponent (+896) and
//    places its 23 fraction bits at the top of the 52; +-0 maps to +-0; subnormals, inf
//    and NaN (rare here) take the hardware conversion.
//  * narrow: round to nearest, ties to even, as the hardware conversion: keep the top
//    23 fraction bits and add one unit when the 29 dropped bits exceed half a unit, or
//    equal it with an odd kept part (a carry into the exponent is the correct rounding,
//    up to infinity past the largest float).  Results below 2^-150 in magnitude round
//    to +-0; results in the binary32 subnormal range, inf and NaN take the hardware
//    conversion.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#ifndef __CUDA_ARCH__
#include <cstring>
#endif

namespace agents {

__host__ __device__ __forceinline__ uint32_t f32_bits(float x) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(x);
#else
  uint32_t b;
  std::memcpy(&b, &x, 4);
  return b;
#endif
}
__host__ __device__ __forceinline__ float f32_from(uint32_t b) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(b);
#else
  float x;
  std::memcpy(&x, &b, 4);
  return x;
#endif
}
__host__ __device__ __forceinline__ uint64_t f64_bits(double x) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(x);
#else
  uint64_t b;
  std::memcpy(&b, &x, 8);
  return b;
#endif
}
__host__ __device__ __forceinline__ double f64_from(uint32_t hi, uint32_t lo) {
#ifdef __CUDA_ARCH__
  return __hiloint2double((int)hi, (int)lo);
#else
  const uint64_t b = ((uint64_t)hi << 32) | lo;
  double x;
  std::memcpy(&x, &b, 8);
  return x;
#endif
}

// Exact float32 -> float64.
__host__ __device__ __forceinline__ double widen(float x) {
  const uint32_t b = f32_bits(x);
  const uint32_t e = (b >> 23) & 0xffu;
  if (e - 1u >= 254u) {                                   // e = 0 or e = 255
    if ((b & 0x7fffffffu) == 0u) return f64_from(b & 0x80000000u, 0u);
    return (double)x;
  }
  return f64_from((b & 0x80000000u) | ((e + 896u) << 20) | ((b >> 3) & 0xfffffu), b << 29);
}

// float64 -> float32, round to nearest, ties to even.
__host__ __device__ __forceinline__ float narrow(double x) {
  const uint64_t b = f64_bits(x);
  const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
  const uint32_t e = (hi >> 20) & 0x7ffu;
  const uint32_t sign = hi & 0x80000000u;
  if (e - 897u > 253u) {                                  // not a normal binary32 result
    if (e <= 872u) return f32_from(sign);                 // |x| < 2^-150 (or 0): +-0
    return (float)x;
  }
  const uint32_t kept = ((hi & 0xfffffu) << 3) | (lo >> 29);
  const uint32_t rest = lo & 0x1fffffffu, half = 0x10000000u;
  const uint32_t up = (rest > half) | ((rest == half) & (kept & 1u));
  return f32_from((sign | ((e - 896u) << 23) | kept) + up);
}

}  // namespace agents
