// FP64 conversions and tests with integer operations (sm_103a): the data
// preparation and the one-pass start convert tens of millions of values,
// and conversions to and from FP64 run on the narrow FP64 pipe of this part.
#pragma once
#include <cuda_runtime.h>

#include <cstring>

namespace concord {

// Bit casts: the device intrinsics, or memcpy in host code (so that the
// host can check these functions against its own conversions).
__host__ __device__ __forceinline__ unsigned fb_f2u(float f) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(f);
#else
  unsigned u;
  std::memcpy(&u, &f, sizeof u);
  return u;
#endif
}
__host__ __device__ __forceinline__ float fb_u2f(unsigned u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float f;
  std::memcpy(&f, &u, sizeof f);
  return f;
#endif
}
__host__ __device__ __forceinline__ unsigned long long fb_d2u(double d) {
#ifdef __CUDA_ARCH__
  return (unsigned long long)__double_as_longlong(d);
#else
  unsigned long long u;
  std::memcpy(&u, &d, sizeof u);
  return u;
#endif
}
__host__ __device__ __forceinline__ double fb_u2d(unsigned long long u) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)u);
#else
  double d;
  std::memcpy(&d, &u, sizeof d);
  return d;
#endif
}

// FP32 -> FP64 widening from the IEEE 754 binary32 / binary64 formats with
// integer operations: a normal number keeps its sign and significand (23 bits
// moved up by 29) and its exponent is rebiased from 127 to 1023, so the result
// is exact and bit-identical to the conversion instruction.  Zeros map to
// signed zeros; subnormals, infinities and NaNs take the conversion
// instruction.  Conversions to and from FP64 run on the narrow FP64 pipe of
// this part, the integer operations do not.
__host__ __device__ __forceinline__ double widen_f32(float f) {
  const unsigned u = fb_f2u(f);
  const unsigned e = (u >> 23) & 0xffu;
  const unsigned long long sgn = (unsigned long long)(u >> 31) << 63;
  if ((u << 1) == 0u) return fb_u2d(sgn);
  if (e == 0u || e == 0xffu) return (double)f;
  return fb_u2d(sgn | ((unsigned long long)(e + 896u) << 52) |
                ((unsigned long long)(u & 0x7fffffu) << 29));
}

__host__ __device__ __forceinline__ double to_f64(double v) { return v; }
__host__ __device__ __forceinline__ double to_f64(float v) { return widen_f32(v); }

// FP64 -> FP32 rounding to nearest (ties to even) with integer operations
// for results in the FP32 normal range: the exponent is rebiased from 1023 to
// 127, the significand keeps its top 23 bits and is rounded on the 29 bits
// dropped; a carry out of the significand moves into the exponent (up to
// infinity past the largest float), as IEEE 754 rounding does.  Inputs below
// the normal range (subnormal or zero results), infinities and NaNs take the
// conversion instruction.  Bit-identical to cvt.rn.f32.f64.
__host__ __device__ __forceinline__ float narrow_f64(double d) {
  const unsigned long long u = fb_d2u(d);
  const unsigned e = (unsigned)(u >> 52) & 0x7ffu;
  if (e < 897u || e > 1150u) return (float)d;
  const unsigned long long m = u & 0xfffffffffffffull;
  unsigned f = ((unsigned)(u >> 63) << 31) | ((e - 896u) << 23) | (unsigned)(m >> 29);
  const unsigned rem = (unsigned)(m & 0x1fffffffull);
  if (rem > 0x10000000u || (rem == 0x10000000u && (f & 1u))) ++f;
  return fb_u2f(f);
}

// isfinite on the bit pattern (exponent field not all ones), integer only.
__host__ __device__ __forceinline__ bool finite_bits(double v) {
  return ((fb_d2u(v) >> 52) & 0x7ffu) != 0x7ffu;
}

}  // namespace concord
