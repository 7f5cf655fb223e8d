// binary64 <-> binary32 conversion by integer operations on the bit fields. On GB300 the
// binary64 pipe issues about two operations per SM and clock; element-wise kernels that
// only need binary32 arithmetic convert with these instead.
#pragma once
#include <cuda_runtime.h>

namespace mlcc {

// truncating binary64 -> binary32; magnitudes below the binary32 normal range give 0,
// NaN and values beyond the range give Inf
__device__ __forceinline__ float d2f_bits(double x) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
  const unsigned hi = unsigned(b >> 32), lo = unsigned(b);
  const int e = int((hi >> 20) & 0x7FF) - 896;   // binary32 biased exponent
  unsigned r = hi & 0x80000000u;
  if (e >= 255) r |= 0x7F800000u;
  else if (e > 0) r |= (unsigned(e) << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29);
  return __uint_as_float(r);
}
// binary64 -> binary32 rounded to nearest (ties to even); magnitudes below the binary32
// normal range give 0, values that round beyond it give Inf, NaN stays NaN
__device__ __forceinline__ float d2f_rn_bits(double x) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
  const unsigned sign = unsigned(b >> 32) & 0x80000000u;
  const int ef = int((b >> 52) & 0x7FF);
  const unsigned long long m = b & ((1ull << 52) - 1);
  if (ef == 0x7FF) return __uint_as_float(sign | 0x7F800000u | (m ? 0x400000u : 0u));
  const int e = ef - 896;   // binary32 biased exponent
  if (e >= 255) return __uint_as_float(sign | 0x7F800000u);
  if (e <= 0) return __uint_as_float(sign);
  unsigned r = (unsigned(e) << 23) | unsigned(m >> 29);
  const unsigned rest = unsigned(m & 0x1FFFFFFFull);
  if (rest > 0x10000000u || (rest == 0x10000000u && (r & 1u))) ++r;   // a carry may reach Inf
  return __uint_as_float(sign | r);
}
// exact binary32 -> binary64 (binary32 subnormals give 0)
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const int e = int((u >> 23) & 0xFF);
  unsigned long long r = static_cast<unsigned long long>(u & 0x80000000u) << 32;
  const unsigned long long m = static_cast<unsigned long long>(u & 0x7FFFFFu) << 29;
  if (e == 255) r |= 0x7FF0000000000000ull | m;
  else if (e > 0) r |= (static_cast<unsigned long long>(e + 896) << 52) | m;
  return __longlong_as_double(static_cast<long long>(r));
}

}  // namespace mlcc
