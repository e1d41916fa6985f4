// Conversions between binary64 and binary32 in integer arithmetic.  GB300's FP64 pipe,
// which the hardware conversions use, runs at about 1/64 of its FP32 rate; kernels that
// convert many values (staging complex128 inputs, forming FP64 outputs from FP32 pairs)
// would be bound by it.  Both follow IEEE 754.  The narrowing hands the cases outside the
// normal binary32 range to the hardware conversion; the widening handles every case
// itself.
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

// binary32 -> binary64, exact, in integer arithmetic for every input: normal numbers have
// their exponent rebased and the fraction widened; subnormals are normalized (the leading
// one found by counting zeros); zeros keep their sign; infinities and NaNs keep the
// all-ones exponent and the widened fraction, NaNs made quiet.  No instruction of it runs
// on the FP64 pipe.
__device__ __forceinline__ double f32_to_f64(float x) {
  const uint32_t b = __float_as_uint(x), sgn = b & 0x80000000u, e = (b >> 23) & 0xFFu, f = b & 0x7FFFFFu;
  uint32_t hi, frac;
  if (e == 0xFFu) {
    frac = f;
    hi = sgn | 0x7FF00000u | (f ? 0x00080000u : 0u);
  } else if (e != 0u) {
    frac = f;
    hi = sgn | ((e + 896u) << 20);
  } else if (f != 0u) {
    const uint32_t p = 31u - (uint32_t)__clz(f);      // the value is f 2^-149 = 1.m 2^(p - 149)
    frac = (f << (23u - p)) & 0x7FFFFFu;
    hi = sgn | ((p + 874u) << 20);
  } else {
    frac = 0u;
    hi = sgn;
  }
  return __hiloint2double((int)(hi | (frac >> 3)), (int)(frac << 29));
}

}  // namespace lhc
