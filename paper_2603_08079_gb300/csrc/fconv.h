// Conversions between binary64 and binary32 done with integer instructions.
//
// On this GPU the float<->double conversion instructions are issued to the
// FP64 unit, which retires about one warp instruction per 19 cycles per SM;
// the mixed-precision kernels convert tens of values per body and are bound
// by that unit.  The conversions below follow the IEEE 754 encodings
// (binary64: 1 sign, 11 exponent bits with bias 1023, 52 fraction bits;
// binary32: 1, 8 with bias 127, 23) and use only integer operations on the
// common path: finite values whose result is a normal binary32 number (or
// zero).  Everything else (subnormal results, overflow, infinities, NaN)
// takes the conversion instruction.
//   f2d: exact (every binary32 value is a binary64 value);
//   d2f: round to nearest, ties to even, the rounding of a C cast.
// The header compiles for the host too (bit copies through memcpy), so that
// the integer paths are tested against the host's own conversions.
#pragma once
#include <stdint.h>
#include <string.h>

#ifdef __CUDACC__
#define MABD_FC __host__ __device__ __forceinline__
#else
#define MABD_FC inline
#endif

namespace mabd {

MABD_FC uint64_t fc_bits64(double x) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(x);
#else
  uint64_t u;
  memcpy(&u, &x, 8);
  return u;
#endif
}

MABD_FC double fc_double(uint32_t hi, uint32_t lo) {
#ifdef __CUDA_ARCH__
  return __hiloint2double((int)hi, (int)lo);
#else
  const uint64_t u = ((uint64_t)hi << 32) | lo;
  double x;
  memcpy(&x, &u, 8);
  return x;
#endif
}

MABD_FC uint32_t fc_bits32(float x) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(x);
#else
  uint32_t u;
  memcpy(&u, &x, 4);
  return u;
#endif
}

MABD_FC float fc_float(uint32_t u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float x;
  memcpy(&x, &u, 4);
  return x;
#endif
}

// binary32 -> binary64 (exact).  Exponent e (1..254) becomes e + 896, the 23
// fraction bits become the top of the 52; zero keeps its sign.  The rare
// cases stay behind a branch: a select would make the compiler issue the
// conversion instruction for every value.
MABD_FC double f2d(float x) {
  const uint32_t u = fc_bits32(x);
  const uint32_t e = (u >> 23) & 0xffu;
  if (e == 0xffu || (e == 0 && (u & 0x7fffffu) != 0)) return (double)x;  // inf, NaN, subnormal
  const uint32_t sign = u & 0x80000000u;
  if (e == 0) return fc_double(sign, 0u);                                 // signed zero
  return fc_double(sign | ((e + 896u) << 20) | ((u >> 3) & 0xfffffu), u << 29);
}

// binary64 -> binary32, round to nearest, ties to even.  For a binary64
// exponent e in 897..1150 the result is a normal binary32 number (or rounds
// up to infinity): the kept 23 fraction bits are the top of the 52, and the
// 29 dropped bits plus 0x0fffffff plus the kept last bit carry exactly when
// they exceed half an ulp or equal it with the last bit odd; a carry out of
// the fraction bumps the exponent.  Zeros keep their sign; the rest
// (subnormal results, |x| >= 2^128, NaN) takes the conversion instruction.
MABD_FC float d2f(double x) {
  const uint64_t u = fc_bits64(x);
  const uint32_t hi = (uint32_t)(u >> 32), lo = (uint32_t)u;
  const uint32_t e = (hi >> 20) & 0x7ffu;
  const uint32_t sign = hi & 0x80000000u;
  if (e == 0 && ((hi & 0xfffffu) | lo) == 0) return fc_float(sign);       // signed zero
  if (e - 897u > 253u) return (float)x;  // result not a normal binary32 number, inf, NaN
  uint32_t f = sign | ((e - 896u) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
  f += ((lo & 0x1fffffffu) + 0x0fffffffu + (f & 1u)) >> 29;
  return fc_float(f);
}

// a binary64 value in the working type T (double or float), and back
template <typename T>
MABD_FC T from_f64(double x);
template <>
MABD_FC double from_f64<double>(double x) { return x; }
template <>
MABD_FC float from_f64<float>(double x) { return d2f(x); }
MABD_FC double to_f64(double x) { return x; }
MABD_FC double to_f64(float x) { return f2d(x); }

}  // namespace mabd
