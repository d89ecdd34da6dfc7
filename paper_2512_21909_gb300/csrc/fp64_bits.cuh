// fp64_bits.cuh -- FP32 -> FP64 conversion with a power-of-two scale, built
// from the bit pattern with integer operations.
//
// GB300 issues 2 FP64 operations per clock per SM, so a tensor-core
// epilogue that converts every FP32 accumulator to FP64 on the FP64 pipe
// (and scales it there) spends more time on the conversions than on the
// MMAs of a short-K product.  The conversion of a normal FP32 number is
// exact and needs only its exponent rebiased and its mantissa shifted; a
// power-of-two scale is an exponent addition.  Zero keeps its sign; FP32
// subnormals, infinities, NaN and results outside the FP64 normal range take
// the arithmetic route (ldexp), so every result equals ldexp((double)x, sh).
#pragma once
#include <cstdint>

namespace cdcc {

// the rare cases, kept out of line so that the unrolled epilogue loops stay
// small
static __device__ __noinline__ double f32_to_f64_slow(float x, int sh) {
  return ldexp((double)x, sh);
}

__device__ __forceinline__ double f32_to_f64_scaled(float x, int sh) {
  const uint32_t f = __float_as_uint(x);
  const int e = (int)((f >> 23) & 0xffu);
  const uint32_t m = f & 0x7fffffu;
  if (e == 0 && m == 0)
    return __longlong_as_double((long long)((uint64_t)(f >> 31) << 63));
  const int E = e - 127 + 1023 + sh;
  if (e == 0 || e == 0xff || E <= 0 || E >= 2047)
    return f32_to_f64_slow(x, sh);
  const uint64_t b = ((uint64_t)(f >> 31) << 63) | ((uint64_t)E << 52) |
                     ((uint64_t)m << 29);
  return __longlong_as_double((long long)b);
}

// alpha as (power-of-two flag, exponent, sign) for the epilogues: a scale
// by +-2^k is folded into the conversion exponent instead of a multiply
struct Pow2 {
  int ok, sh, neg;
};

inline Pow2 pow2_of(double a) {
  Pow2 p{0, 0, 0};
  if (!(a != 0.0) || a != a) return p;
  int ex = 0;
  const double m = std::frexp(a, &ex);   // a = m * 2^ex, 0.5 <= |m| < 1
  if (m == 0.5 || m == -0.5) {
    p.ok = 1;
    p.sh = ex - 1;
    p.neg = m < 0 ? 1 : 0;
  }
  return p;
}

}  // namespace cdcc
