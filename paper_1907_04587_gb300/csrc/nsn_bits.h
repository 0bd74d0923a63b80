// Bit-level arithmetic shared by host and device: an exact binary32 ->
// binary64 conversion with integer operations only, and the double-word
// binary32 evaluation of the CR recurrence ApTPAp = d2 + 2 beta d3 + beta^2 d5.
//
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

#include <math.h>
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

// Correctly rounded binary32 operations, never contracted: the CUDA
// round-to-nearest intrinsics on the device, plain operations (compiled
// without contraction, as ISO C does) and fmaf on the host.
NSN_BITS_HD float nsn_add_rn(float a, float b) {
#if defined(__CUDA_ARCH__)
  return __fadd_rn(a, b);
#else
  return a + b;
#endif
}
NSN_BITS_HD float nsn_mul_rn(float a, float b) {
#if defined(__CUDA_ARCH__)
  return __fmul_rn(a, b);
#else
  return a * b;
#endif
}
NSN_BITS_HD float nsn_fma_rn(float a, float b, float c) {
#if defined(__CUDA_ARCH__)
  return __fmaf_rn(a, b, c);
#else
  return fmaf(a, b, c);
#endif
}

// Error-free transformations: a + b = s + e exactly (Knuth's TwoSum), and
// a b = p + e exactly (the FMA form of TwoProduct, Ogita, Rump and Oishi,
// "Accurate sum and dot product", 2005), barring overflow and underflow.
NSN_BITS_HD void nsn_two_sum(float a, float b, float *s, float *e) {
  const float ss = nsn_add_rn(a, b);
  const float bb = nsn_add_rn(ss, -a);
  *s = ss;
  *e = nsn_add_rn(nsn_add_rn(a, -nsn_add_rn(ss, -bb)), nsn_add_rn(b, -bb));
}
NSN_BITS_HD void nsn_two_prod(float a, float b, float *p, float *e) {
  const float pp = nsn_mul_rn(a, b);
  *p = pp;
  *e = nsn_fma_rn(a, b, -pp);
}

// ApTPAp = d2 + 2 beta d3 + beta^2 d5 of binary32 terms, carried in two
// binary32 words and rounded once: 2 beta d3 = ph + pl and beta^2 = bh + bl
// exactly, bh d5 exactly, bl d5 with one rounding (2^-48 of that term); the
// sums by TwoSum, their error terms added in binary32.  The cancellation of
// the recurrence then costs about what it costs in binary64 (a 48-bit
// significand against 53), on the binary32 pipes.
NSN_BITS_HD float nsn_apap_f32(float d2, float d3, float d5, float beta) {
  float ph, pl, bh, bl, qh, ql, s, e, s2, e2;
  nsn_two_prod(beta, d3, &ph, &pl);
  ph = nsn_mul_rn(2.0f, ph);
  pl = nsn_mul_rn(2.0f, pl);   /* exact */
  nsn_two_prod(beta, beta, &bh, &bl);
  nsn_two_prod(bh, d5, &qh, &ql);
  ql = nsn_fma_rn(bl, d5, ql);
  nsn_two_sum(d2, ph, &s, &e);
  nsn_two_sum(s, qh, &s2, &e2);
  return nsn_add_rn(s2, nsn_add_rn(nsn_add_rn(e, pl), nsn_add_rn(e2, ql)));
}
