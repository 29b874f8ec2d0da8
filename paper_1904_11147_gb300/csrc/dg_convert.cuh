// Conversions that keep the FP64 pipe free.
#pragma once

namespace dg {

// double -> float by truncation of the significand on the integer pipe (keeps the FP64
// pipe, the bottleneck of the method on GB300, free): relative error below 2^-23; values
// below the float range give 0, values above it (and NaN) give an infinity.
__device__ __forceinline__ float d2f_trunc(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned int sign = (unsigned int)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7ff) - 1023 + 127;
  if (e <= 0) return __uint_as_float(sign);
  if (e >= 255) return __uint_as_float(sign | 0x7f800000u);
  return __uint_as_float(sign | ((unsigned int)e << 23) | (unsigned int)((b >> 29) & 0x7fffffu));
}

}  // namespace dg
