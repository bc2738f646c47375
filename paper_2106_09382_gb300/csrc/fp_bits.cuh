// FP64 conversions and tests with integer operations (sm_103a): the data
// preparation and the one-pass start convert tens of millions of values,
// and conversions to and from FP64 run on the narrow FP64 pipe of this part.
#pragma once
#include <cuda_runtime.h>

namespace concord {

// FP32 -> FP64 widening from the IEEE 754 binary32 / binary64 formats with
// integer operations: a normal number keeps its sign and significand (23 bits
// moved up by 29) and its exponent is rebiased from 127 to 1023, so the result
// is exact and bit-identical to the conversion instruction.  Zeros map to
// signed zeros; subnormals, infinities and NaNs take the conversion
// instruction.  Conversions to and from FP64 run on the narrow FP64 pipe of
// this part, the integer operations do not.
__device__ __forceinline__ double widen_f32(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu;
  const unsigned long long sgn = (unsigned long long)(u >> 31) << 63;
  if ((u << 1) == 0u) return __longlong_as_double((long long)sgn);
  if (e == 0u || e == 0xffu) return (double)f;
  return __longlong_as_double((long long)(sgn | ((unsigned long long)(e + 896u) << 52) |
                                          ((unsigned long long)(u & 0x7fffffu) << 29)));
}

__device__ __forceinline__ double to_f64(double v) { return v; }
__device__ __forceinline__ double to_f64(float v) { return widen_f32(v); }

// isfinite on the bit pattern (exponent field not all ones), integer only.
__device__ __forceinline__ bool finite_bits(double v) {
  return ((__double_as_longlong(v) >> 52) & 0x7ff) != 0x7ff;
}

}  // namespace concord
