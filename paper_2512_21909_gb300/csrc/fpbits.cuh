// fpbits.cuh -- FP64 values formed with integer operations.
//
// GB300 executes FP64 at 2 DFMA per clock per SM; an epilogue that converts
// and scales every output element in FP64 can cost more than the
// tensor-core work of a short-K tile.  f2d_pow2 builds the double f * 2^k
// of a float from its bit pattern (bitwise equal to ldexp((double)f, k));
// zeros stay on the integer path, subnormal, infinite or NaN inputs and
// results outside the normal range take the FP64 path.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace cdcc {

__device__ __forceinline__ double f2d_pow2(float f, int k) {
  const uint32_t u = __float_as_uint(f);
  const unsigned long long sign = (unsigned long long)(u >> 31) << 63;
  if ((u << 1) == 0u) return __longlong_as_double((long long)sign);
  const int e8 = (int)((u >> 23) & 0xffu);
  const int e11 = e8 - 127 + 1023 + k;
  if (e8 == 0 || e8 == 255 || e11 <= 0 || e11 >= 2047)
    return ldexp((double)f, k);
  const unsigned long long bits =
      sign | ((unsigned long long)e11 << 52) |
      ((unsigned long long)(u & 0x7fffffu) << 29);
  return __longlong_as_double((long long)bits);
}

}  // namespace cdcc
