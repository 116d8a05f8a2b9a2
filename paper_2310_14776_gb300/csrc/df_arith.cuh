// df_arith.cuh -- double-float arithmetic helpers: a value carried as the unevaluated sum
// hi + lo of two FP32 numbers (about 48 significant bits).  GB300 issues about two FP64 FMAs
// per SM and clock, 1/64 of its FP32 rate, so FP64-accurate work that the FP64 pipe would
// bound runs faster on the FP32 pipe in this form.  Conversions to and from FP64 use integer
// operations on the IEEE fields, off the FP64 pipe.
#pragma once

#include <cuda_runtime.h>

namespace pawfd {
namespace dfa {

struct __align__(8) DF {
  float hi, lo;
};

// The rare path of split64, kept out of line: inlined, the compiler evaluates it for every
// value under a predicate, and its three FP64 conversions and one FP64 subtraction per value
// then fill the narrow FP64 pipe (ncu showed the pipe 75 % busy for what should be one
// addition per stencil point).
static __device__ __noinline__ DF split64_slow(double x) {
  const float hi = __double2float_rn(x);
  return {hi, __double2float_rn(x - (double)hi)};
}

// x = hi + lo: hi = x rounded to 24 bits, lo = x - hi rounded to 24 bits (so hi + lo equals x
// to a relative 2^-48).  The IEEE fields are split with integer operations; values outside
// the normal FP32 range of both parts take the conversion path.
__device__ __forceinline__ DF split64(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned h = (unsigned)(b >> 32), l = (unsigned)b;
  const int e = (int)((h >> 20) & 0x7FFu);
  if (e < 960 || e > 1140) return split64_slow(x);
  const unsigned top = (((h & 0xFFFFFu) | 0x100000u) << 3) | (l >> 29);   // 24-bit significand
  const unsigned rem = l & 0x1FFFFFFFu;                                    // the 29 bits below
  const unsigned up = rem >> 28;                                           // round half up
  // exponent (e - 1023 + 127) and the 23 stored bits; a carry of the rounding runs into the
  // exponent, as it must
  const unsigned hbits = (h & 0x80000000u) | ((((unsigned)(e - 896)) << 23) + (top & 0x7FFFFFu) + up);
  // residual in units of 2^(e - 1075): rem - up 2^29, |r| <= 2^28
  const int r = (int)rem - (int)(up << 29);
  const float scale = __int_as_float((e - 948) << 23);                     // 2^(e - 1075)
  float lo = __int2float_rn(r) * scale;
  if (h & 0x80000000u) lo = -lo;
  return {__uint_as_float(hbits), lo};
}

// exact float -> double from the IEEE fields (integer operations only); zero and subnormal
// inputs give zero (below 2^-126, far under the 2^-48 relative accuracy of the pairs)
__device__ __forceinline__ double f2d(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xFFu;
  if (e == 0) return 0.0;
  const unsigned long long b = ((unsigned long long)(u & 0x80000000u) << 32) |
                               ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)(u & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)b);
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// acc += a b for pairs, keeping acc normalized (|lo| <= ulp(hi) / 2): the product's rounding
// errors enter lo through FMAs (the lo x lo term, below 2^-48 of the product, is dropped), the
// sum of the high parts is error-free (TwoSum), and a final fast TwoSum renormalizes, so each
// step adds a relative error of order 2^-47 of |acc|.
__device__ __forceinline__ void fma_acc(DF& acc, DF a, DF b) {
  const float ph = a.hi * b.hi;
  float pe = fmaf(a.hi, b.hi, -ph);
  pe = fmaf(a.hi, b.lo, pe);
  pe = fmaf(a.lo, b.hi, pe);
  float s, e;
  two_sum(acc.hi, ph, s, e);
  e += acc.lo + pe;
  acc.hi = s + e;
  acc.lo = e - (acc.hi - s);
}

__device__ __forceinline__ double to_double(DF x) { return f2d(x.hi) + f2d(x.lo); }

}  // namespace dfa
}  // namespace pawfd
