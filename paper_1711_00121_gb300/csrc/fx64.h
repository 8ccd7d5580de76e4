// Exact sums of FP64 values in 64-bit fixed point on the integer pipe, and
// their rounding back to FP64.
//
// GB300 issues FP64 instructions at 1/64 of the FP32 rate, and a warp pays for
// an FP64 instruction whichever of its lanes use it, so the pre-update
// kernel forms its row sums of FP64 vector entries here:
//   - every value v of a group (the values of one row held by a run of lanes)
//     becomes fx_of(v, em) = v * 2^(1078 - em) truncated toward zero, where em
//     is the largest biased exponent in the group: |fx| < 2^56, an error below
//     2^(em - 1078), i.e. 2^-55 of the group's largest value;
//   - up to 128 such numbers add exactly in a signed 64-bit integer;
//   - fx_value(t, em) = t * 2^(em - 1078) rounded once to FP64 (one integer to
//     FP64 conversion; the power of two goes into the exponent field).
// Values that are zero or subnormal count as zero (fx_exp returns 0).
#pragma once

#include <cmath>
#include <cstdint>

#if defined(__CUDACC__)
#define FX_HD __host__ __device__ __forceinline__
#else
#define FX_HD inline
#endif

namespace sr {

FX_HD uint64_t fx_bits(double v) {
#if defined(__CUDA_ARCH__)
  return (uint64_t)__double_as_longlong(v);
#else
  uint64_t b;
  __builtin_memcpy(&b, &v, 8);
  return b;
#endif
}

FX_HD double fx_from_bits(uint64_t b) {
#if defined(__CUDA_ARCH__)
  return __longlong_as_double((long long)b);
#else
  double v;
  __builtin_memcpy(&v, &b, 8);
  return v;
#endif
}

// biased binary exponent of v (0 for zero and subnormal values)
FX_HD int fx_exp(double v) { return (int)((fx_bits(v) >> 52) & 0x7ff); }

// v * 2^(1078 - em) truncated toward zero, for fx_exp(v) <= em
FX_HD int64_t fx_of(double v, int em) {
  const uint64_t b = fx_bits(v);
  const int ex = (int)((b >> 52) & 0x7ff);
  if (ex == 0) return 0;
  const uint64_t m = (b & 0xfffffffffffffull) | 0x10000000000000ull;  // 53-bit significand
  const int sh = ex - em + 3;  // v * 2^(1078 - em) = m * 2^sh, sh <= 3
  const uint64_t f = sh >= 0 ? (m << sh) : (sh > -54 ? (m >> -sh) : 0ull);
  return (int64_t)(b >> 63) ? -(int64_t)f : (int64_t)f;
}

// t * 2^(em - 1078) rounded once to FP64 (the conversion of t rounds; the
// power of two is added to the exponent field when the result stays normal,
// else applied by ldexp)
FX_HD double fx_value(int64_t t, int em) {
  if (t == 0) return 0.0;
  const double d = (double)t;  // |t| < 2^63: one rounding
  if (em >= 56 && em < 1960)
    return fx_from_bits(fx_bits(d) + ((uint64_t)(int64_t)(em - 1078) << 52));
  return ldexp(d, em - 1078);
}

}  // namespace sr
