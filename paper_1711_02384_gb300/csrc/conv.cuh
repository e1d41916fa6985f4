// Conversions between binary64 and binary32 in integer arithmetic.  GB300's FP64 pipe,
// which the hardware conversions use, runs at about 1/64 of its FP32 rate; kernels that
// convert many values (staging complex128 inputs, forming FP64 outputs from FP32 pairs)
// would be bound by it.  Both functions follow IEEE 754 for the cases they handle and
// hand every other case (zero, subnormals, infinities, NaN, out-of-range) to the
// hardware conversion.
#pragma once

#include <stdint.h>

namespace lhc {

// binary64 -> binary32, round to nearest even.  For results in the normal binary32 range
// the exponent is rebased, the top 23 fraction bits are kept and the 29 dropped bits
// round the result (a carry into the exponent is the correct rounding, up to infinity).
__device__ __forceinline__ float f64_to_f32_rne(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const uint32_t hi = (uint32_t)(u >> 32), lo = (uint32_t)u;
  const uint32_t ahi = hi & 0x7FFFFFFFu, e = ahi >> 20;
  if (e < 897u || e >= 1151u) return __double2float_rn(x);
  uint32_t f = ((ahi - (896u << 20)) << 3) | (lo >> 29);
  f += ((lo & 0x1FFFFFFFu) + (f & 1u) + 0x0FFFFFFFu) >> 29;
  return __uint_as_float((hi & 0x80000000u) | f);
}

// binary32 -> binary64, exact: the exponent is rebased and the fraction widened.
__device__ __forceinline__ double f32_to_f64(float x) {
  const uint32_t b = __float_as_uint(x), e = (b >> 23) & 0xFFu;
  if (e == 0u || e == 0xFFu) return (double)x;
  const uint32_t hi = (b & 0x80000000u) | ((e + 896u) << 20) | ((b & 0x7FFFFFu) >> 3);
  return __hiloint2double((int)hi, (int)(b << 29));
}

}  // namespace lhc
