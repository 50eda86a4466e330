// FP32 -> FP64 widening without the FP64 unit (shared by the solver kernels).
#pragma once
#include <cuda_runtime.h>

namespace mlmc {

// Widening of an FP32 value to FP64 on the integer pipe only (GB300's FP64 unit, which
// also performs the hardware conversion, runs at 1/64 of the FP32 rate, and a fallback
// branch to the hardware conversion is if-converted into every call): for normal numbers
// the binary64 pattern is the binary32 sign, the exponent re-biased by 1023 - 127 and the
// 23-bit fraction shifted left by 29 (IEEE 754 layouts), exact; zeros stay zero,
// infinities and NaNs keep an all-ones exponent, subnormals (below 1.2e-38; faces and
// diagonals are positive normal numbers) flush to zero, an absolute change below 1.2e-38.
__device__ __forceinline__ double widen(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned e = (b >> 23) & 0xffu;
  const unsigned hi_e = e == 0u ? 0u : (e == 0xffu ? 0x7ffu : e + (1023u - 127u));
  const unsigned frac = e == 0u ? 0u : (b & 0x7fffffu);
  const unsigned hi = (b & 0x80000000u) | (hi_e << 20) | (frac >> 3);
  const unsigned lo = frac << 29;
  return __hiloint2double((int)hi, (int)lo);
}
__device__ __forceinline__ double widen(double d) { return d; }

// Narrowing of an FP64 value to FP32, round to nearest even, on the integer pipe only:
// the binary32 fraction is the top 23 of the 52 fraction bits, rounded up when the
// remaining 29 bits exceed half an ulp or equal it with an odd result (a carry into the
// exponent is the correct rounding of an all-ones fraction); exponents past the binary32
// range give infinity, results below 2^-126 (1.2e-38) flush to zero; NaNs are not
// expected (the operands are finite residuals).
__device__ __forceinline__ float narrow(double d) {
  const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
  const unsigned sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7ffu) - 1023 + 127;
  unsigned frac = ((hi & 0xfffffu) << 3) | (lo >> 29);
  const unsigned rem = lo & 0x1fffffffu;
  frac += (rem > 0x10000000u || (rem == 0x10000000u && (frac & 1u))) ? 1u : 0u;
  // frac == 2^23 after the carry: the exponent field absorbs it below
  const unsigned body = ((unsigned)e << 23) + frac;
  const unsigned bits = e <= 0 ? sign : (e >= 255 ? (sign | 0x7f800000u) : (sign | (body >= 0x7f800000u ? 0x7f800000u : body)));
  return __uint_as_float(bits);
}

}  // namespace mlmc
