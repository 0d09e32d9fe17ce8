// Double-float arithmetic: a value is the unevaluated sum h + l of two
// binary32 numbers with |l| < ulp(h), about 46 significant bits.
//
// On this GPU an FP64 instruction holds the FP64 unit for about as long as
// 76 FP32 instructions take to issue, and the mixed-precision kernels that
// must reproduce the FP64 system (the rotation, the right-hand side) are
// bound by that unit.  The operations below take 3 to 20 FP32 instructions
// each.  They are built from two error-free transformations: Knuth's
// TwoSum (s = fl(a + b) and the exact error a + b - s, six additions) and
// the product with its exact error from one fused multiply-add
// (a b - fl(a b) is a binary32 number, returned by fma(a, b, -fl(a b))).
// The additions here are the short ("sloppy") form: the error of a sum is
// a few units of 2^-46 of the larger operand, as with binary64 rounding,
// which is 2^-53 of it.
//
// Every operation goes through the round-to-nearest intrinsics on the
// device so that the compiler neither contracts nor reorders them; the
// header compiles for the host as well (tests/native/ff_check.cpp checks
// it against long double).
#pragma once
#include "fconv.h"
#ifndef __CUDA_ARCH__
#include <math.h>
#endif

namespace mabd {

struct ff {
  float h, l;
};

MABD_FC float ff_add1(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fadd_rn(a, b);
#else
  return a + b;
#endif
}

MABD_FC float ff_sub1(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fsub_rn(a, b);
#else
  return a - b;
#endif
}

MABD_FC float ff_mul1(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fmul_rn(a, b);
#else
  return a * b;
#endif
}

MABD_FC float ff_fma1(float a, float b, float c) {
#ifdef __CUDA_ARCH__
  return __fmaf_rn(a, b, c);
#else
  return fmaf(a, b, c);
#endif
}

MABD_FC int ff_msb(uint32_t m) {  // index of the highest set bit of m > 0
#ifdef __CUDA_ARCH__
  return 31 - __clz((int)m);
#else
  return 31 - __builtin_clz(m);
#endif
}

// Knuth's TwoSum: a + b = s + e exactly, s = fl(a + b)
MABD_FC ff two_sum(float a, float b) {
  const float s = ff_add1(a, b);
  const float bb = ff_sub1(s, a);
  const float e = ff_add1(ff_sub1(a, ff_sub1(s, bb)), ff_sub1(b, bb));
  return {s, e};
}

// the same when |a| >= |b| (or a = 0): three additions
MABD_FC ff fast_two_sum(float a, float b) {
  const float s = ff_add1(a, b);
  return {s, ff_sub1(b, ff_sub1(s, a))};
}

// a b = p + e exactly, p = fl(a b)
MABD_FC ff two_prod(float a, float b) {
  const float p = ff_mul1(a, b);
  return {p, ff_fma1(a, b, -p)};
}

MABD_FC ff ff_make(float a) { return {a, 0.0f}; }
MABD_FC ff ff_neg(ff a) { return {-a.h, -a.l}; }

MABD_FC ff ff_add(ff a, ff b) {
  const ff s = two_sum(a.h, b.h);
  return fast_two_sum(s.h, ff_add1(s.l, ff_add1(a.l, b.l)));
}

MABD_FC ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }

MABD_FC ff ff_mul(ff a, ff b) {
  const ff p = two_prod(a.h, b.h);
  float e = ff_fma1(a.h, b.l, p.l);
  e = ff_fma1(a.l, b.h, e);
  return fast_two_sum(p.h, e);
}

MABD_FC ff ff_mulf(ff a, float b) {
  const ff p = two_prod(a.h, b);
  return fast_two_sum(p.h, ff_fma1(a.l, b, p.l));
}

// a b + c with one final normalisation
MABD_FC ff ff_fma(ff a, ff b, ff c) {
  const ff p = two_prod(a.h, b.h);
  float e = ff_fma1(a.h, b.l, p.l);
  e = ff_fma1(a.l, b.h, e);
  const ff s = two_sum(p.h, c.h);
  return fast_two_sum(s.h, ff_add1(s.l, ff_add1(e, c.l)));
}

// 1 / a: the binary32 reciprocal refined by one Newton step, r + r (1 - a r)
MABD_FC ff ff_rcp(ff a) {
  const float r = 1.0f / a.h;
  const ff e = ff_sub(ff_make(1.0f), ff_mulf(a, r));
  return ff_add(ff_make(r), ff_mulf(e, r));
}

// binary64 -> double-float with integer instructions: h is x cut to its
// leading 24 significant bits and l the rest (the 29 dropped fraction bits,
// of x's sign) cut to its leading 24; both are normal binary32 numbers for
// binary64 exponents e in 950..1140 (|x| in [2^-73, 2^118)); zeros keep
// their sign.  Other values (tiny, huge, non-finite) take the conversion
// instructions.
// (kept out of line: inlined, the compiler may evaluate its conversions for
// every value instead of branching around them)
#ifdef __CUDA_ARCH__
__device__ __noinline__
#else
inline
#endif
ff ff_from_rare(double x) {
  const float h = (float)x;
  const double r = x - (double)h;
  return {h, r == r ? (float)r : 0.0f};  // infinities and NaN: l = 0
}

MABD_FC ff ff_from(double x) {
  const uint64_t u = fc_bits64(x);
  const uint32_t hi = (uint32_t)(u >> 32), lo = (uint32_t)u;
  const uint32_t e = (hi >> 20) & 0x7ffu;
  if (e - 950u > 190u) {
    if ((u << 1) == 0) return {fc_float(hi), 0.0f};  // signed zero
    return ff_from_rare(x);
  }
  const uint32_t sign = hi & 0x80000000u;
  const float h = fc_float(sign | ((e - 896u) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29));
  const uint32_t m = lo & 0x1fffffffu;
  if (m == 0) return {h, 0.0f};
  // the rest is m 2^(e - 1075); with its top bit at p it is a binary32
  // number of exponent field p + e - 948
  const int p = ff_msb(m);
  const uint32_t frac = (p >= 23 ? (m >> (p - 23)) : (m << (23 - p))) & 0x7fffffu;
  return {h, fc_float(sign | ((uint32_t)(p + (int)e - 948) << 23) | frac)};
}

// double-float -> binary64 (one binary64 addition)
MABD_FC double ff_to(ff a) { return f2d(a.h) + f2d(a.l); }

}  // namespace mabd
