// Exact binary32 -> binary64 conversion with integer operations only.
//
// The value of a binary32 number is carried over unchanged into binary64
// (IEEE 754: every binary32 value is a binary64 value), so the conversion is
// a re-encoding of the fields: the sign bit moves to bit 63, a normal
// exponent is re-biased from 127 to 1023 (an addition of 896), the 23-bit
// fraction is shifted up by 29 bits; zeros stay zeros, infinities and NaNs
// keep an all-ones exponent (the NaN payload shifted like a fraction); a
// subnormal m * 2^-149 becomes the normal number whose leading one is m's
// highest set bit p: exponent p - 149 + 1023, fraction m without that bit,
// shifted to the top of the 52-bit field.
//
// On GB300 the hardware conversion instruction runs on the narrow FP64 pipe
// (a warp-wide instruction occupies it for many cycles); this form uses the
// integer pipe.  Host and device share the code; the host build is what the
// CPU test checks against the C conversion.
#pragma once

#include <stdint.h>
#include <string.h>

#if defined(__CUDACC__)
#define NSN_BITS_HD __host__ __device__ __forceinline__
#else
#define NSN_BITS_HD static inline
#endif

NSN_BITS_HD uint32_t nsn_bits_f32(float x) {
#if defined(__CUDA_ARCH__)
  return __float_as_uint(x);
#else
  uint32_t u;
  memcpy(&u, &x, sizeof u);
  return u;
#endif
}

NSN_BITS_HD double nsn_f64_from_bits(uint64_t d) {
#if defined(__CUDA_ARCH__)
  return __longlong_as_double((long long)d);
#else
  double x;
  memcpy(&x, &d, sizeof x);
  return x;
#endif
}

// index of the highest set bit of a nonzero 32-bit value
NSN_BITS_HD int nsn_bits_top(uint32_t m) {
#if defined(__CUDA_ARCH__)
  return 31 - __clz((int)m);
#else
  return 31 - __builtin_clz(m);
#endif
}

NSN_BITS_HD double nsn_f32_to_f64_exact(float x) {
  const uint32_t u = nsn_bits_f32(x);
  const uint64_t s = (uint64_t)(u >> 31) << 63;
  const uint32_t e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
  uint64_t d;
  if (e == 0xffu) {
    d = (0x7ffull << 52) | ((uint64_t)m << 29);
  } else if (e != 0u) {
    d = ((uint64_t)(e + 896u) << 52) | ((uint64_t)m << 29);
  } else if (m == 0u) {
    d = 0;
  } else {
    const int p = nsn_bits_top(m);   // 0 .. 22
    d = ((uint64_t)(p + 874) << 52) | ((uint64_t)(m ^ (1u << p)) << (52 - p));
  }
  return nsn_f64_from_bits(s | d);
}
