// IEEE-754 conversions between binary32 and binary64 done with integer
// operations on the bit patterns, so that they run on the integer ALUs rather
// than on GB300's narrow FP64 pipe (the only consumers stream data at the HBM
// rate, where the FP64 pipe, not memory, would otherwise be the limit).
#pragma once

#include <cuda_runtime.h>

namespace lqcd {

// binary32 -> binary64, exact for every input (zeros, subnormals, infinities,
// NaNs keep their sign; NaN payloads are shifted into the wider field).
__host__ __device__ __forceinline__ double f32_to_f64_bits(float f) {
#ifdef __CUDA_ARCH__
  const unsigned u = __float_as_uint(f);
#else
  unsigned u;
  __builtin_memcpy(&u, &f, 4);
#endif
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  const unsigned e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
  unsigned long long bits;
  if (e == 0xffu) {
    bits = sign | 0x7ff0000000000000ull | ((unsigned long long)m << 29);
  } else if (e != 0u) {
    bits = sign | ((unsigned long long)(e + (1023u - 127u)) << 52) | ((unsigned long long)m << 29);
  } else if (m == 0u) {
    bits = sign;
  } else {  // subnormal binary32: value m * 2^-149, leading bit at position p
#ifdef __CUDA_ARCH__
    const int p = 31 - __clz(m);
#else
    const int p = 31 - __builtin_clz(m);
#endif
    const unsigned long long mant = ((unsigned long long)m << (52 - p)) & 0xfffffffffffffull;
    bits = sign | ((unsigned long long)(p - 149 + 1023) << 52) | mant;
  }
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)bits);
#else
  double d;
  __builtin_memcpy(&d, &bits, 8);
  return d;
#endif
}

// binary64 d * 2^e2 -> binary32, rounded to nearest with ties away from zero;
// results below the smallest normal binary32 are flushed to a signed zero,
// results above the largest finite one become infinities, NaNs stay NaNs.  The
// power of two is applied to the exponent field before rounding, so it is exact;
// binary64 subnormal inputs count as zeros.
__host__ __device__ __forceinline__ float f64_to_f32_bits(double d, int e2 = 0) {
#ifdef __CUDA_ARCH__
  const unsigned long long u = (unsigned long long)__double_as_longlong(d);
#else
  unsigned long long u;
  __builtin_memcpy(&u, &d, 8);
#endif
  const unsigned sign = (unsigned)(u >> 32) & 0x80000000u;
  const int e = (int)((u >> 52) & 0x7ffu);
  const unsigned long long m = u & 0xfffffffffffffull;
  unsigned bits;
  if (e == 0x7ff) {
    bits = sign | 0x7f800000u | (m ? 0x400000u : 0u);
  } else {
    const int ef = e == 0 ? 0 : e - 1023 + 127 + e2;
    if (ef >= 255) {
      bits = sign | 0x7f800000u;
    } else if (ef <= 0) {
      bits = sign;
    } else {
      // drop 29 mantissa bits, rounding on the highest dropped one; a carry
      // into the exponent (or up to the infinity pattern) is the correct result
      bits = sign | (unsigned)(((((unsigned long long)ef) << 52 | m) + (1ull << 28)) >> 29);
    }
  }
#ifdef __CUDA_ARCH__
  return __uint_as_float(bits);
#else
  float f;
  __builtin_memcpy(&f, &bits, 4);
  return f;
#endif
}

// s = m * 2^e with m in [1, 2) as a binary32 (rounded to nearest, ties away),
// for a finite normal binary64 s; returns false (e, m untouched) otherwise.
// With it, (float)(d * s) is computed as f64_to_f32_bits(d, e) * m: no FP64 work,
// at most one binary32 rounding more than the direct product.
__host__ __device__ __forceinline__ bool split_pow2(double s, int &e, float &m) {
#ifdef __CUDA_ARCH__
  const unsigned long long u = (unsigned long long)__double_as_longlong(s);
#else
  unsigned long long u;
  __builtin_memcpy(&u, &s, 8);
#endif
  const int ex = (int)((u >> 52) & 0x7ffu);
  if (ex == 0 || ex == 0x7ff) return false;
  e = ex - 1023;
  const unsigned long long one = (u & 0x800fffffffffffffull) | (1023ull << 52);
#ifdef __CUDA_ARCH__
  m = f64_to_f32_bits(__longlong_as_double((long long)one));
#else
  double dm;
  __builtin_memcpy(&dm, &one, 8);
  m = f64_to_f32_bits(dm);
#endif
  return true;
}

}  // namespace lqcd
