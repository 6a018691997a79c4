// Double-float ("ff") arithmetic on the FP32 pipes, for the mixed-precision path.
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2,
// about 48 significand bits.  The building blocks are the error-free
// transformations of Knuth (TwoSum) and Dekker (Fast2Sum; with an FMA, TwoProd
// is p = a*b, e = fma(a, b, -p)); the add and multiply below are the usual
// "sloppy" double-word forms (Dekker 1971; Joldes, Muller and Popescu, ACM TOMS
// 2017), whose error is a few units of 2^-48 of the operand magnitudes.
// GB300 issues FP64 at 1/64 of its FP32 rate, so these ~10-instruction
// operations are several times cheaper than one native FP64 operation, and the
// conversions to and from FP64 below use integer bit manipulation for the same
// reason (FP64<->FP32 conversions run at the FP64 rate).
#pragma once

#include <stdint.h>

namespace chx {

struct ff {
  float hi, lo;
};

// |a| >= |b| (or a == 0)
__device__ __forceinline__ ff fast_two_sum(float a, float b) {
  const float s = a + b;
  return ff{s, b - (s - a)};
}

__device__ __forceinline__ ff two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return ff{s, (a - (s - bb)) + (b - bb)};
}

__device__ __forceinline__ ff two_prod(float a, float b) {
  const float p = a * b;
  return ff{p, fmaf(a, b, -p)};
}

__device__ __forceinline__ ff ff_add(ff x, ff y) {
  ff s = two_sum(x.hi, y.hi);
  return fast_two_sum(s.hi, s.lo + (x.lo + y.lo));
}

__device__ __forceinline__ ff ff_neg(ff x) { return ff{-x.hi, -x.lo}; }

__device__ __forceinline__ ff ff_sub(ff x, ff y) { return ff_add(x, ff_neg(y)); }

__device__ __forceinline__ ff ff_add_f(ff x, float y) {
  ff s = two_sum(x.hi, y);
  return fast_two_sum(s.hi, s.lo + x.lo);
}

__device__ __forceinline__ ff ff_mul(ff x, ff y) {
  ff p = two_prod(x.hi, y.hi);
  float e = fmaf(x.hi, y.lo, p.lo);
  e = fmaf(x.lo, y.hi, e);
  return fast_two_sum(p.hi, e);
}

__device__ __forceinline__ ff ff_mul_f(ff x, float y) {
  ff p = two_prod(x.hi, y);
  return fast_two_sum(p.hi, fmaf(x.lo, y, p.lo));
}

// Exact scaling by a power of two (no rounding barring over/underflow).
__device__ __forceinline__ ff ff_scale2(ff x, float p2) { return ff{x.hi * p2, x.lo * p2}; }

// FP64 -> ff by bit manipulation: hi is the double truncated to 24 significand
// bits, lo the rest rounded to 24 bits (so ~2^-48 relative).  Magnitudes below
// 2^-126 are flushed to zero; lo is dropped below 2^-100 relative reach.
__device__ __forceinline__ ff d2ff(double x) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  const uint32_t sgn = (uint32_t)(b >> 63) << 31;
  const int e = (int)((b >> 52) & 0x7ff);
  const uint64_t m = b & 0xFFFFFFFFFFFFFull;
  const int fe = e - 1023 + 127;
  if (fe <= 0) return ff{__uint_as_float(sgn), 0.f};
  if (e == 0x7ff || fe >= 255) {  // Inf/NaN or out of float range: carry it in hi
    return ff{__uint_as_float(sgn | 0x7f800000u | (m ? 0x400000u : 0u)), 0.f};
  }
  const float hi = __uint_as_float(sgn | ((uint32_t)fe << 23) | (uint32_t)(m >> 29));
  const uint32_t r = (uint32_t)(m & 0x1FFFFFFFull);  // low 29 bits
  float lo = 0.f;
  const int se = e - 1075 + 127;  // exponent of 2^(e - 1075), the weight of r's unit bit
  if (r != 0 && se > 0) {
    lo = __uint2float_rn(r) * __uint_as_float((uint32_t)se << 23);
    if (sgn) lo = -lo;
  }
  return ff{hi, lo};
}

// Exact float -> double by bit manipulation (denormal floats flush to zero).
__device__ __forceinline__ double f2d_exact(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t e = (u >> 23) & 0xff;
  const uint64_t sgn = (uint64_t)(u >> 31) << 63;
  if (e == 0) return __longlong_as_double((long long)sgn);
  if (e == 255) return __longlong_as_double((long long)(sgn | 0x7ff0000000000000ull | ((uint64_t)(u & 0x7fffff) << 29)));
  return __longlong_as_double((long long)(sgn | ((uint64_t)(e + 896) << 52) | ((uint64_t)(u & 0x7fffff) << 29)));
}

// ff -> FP64: both parts convert exactly; one FP64 add rounds the sum.
__device__ __forceinline__ double ff2d(ff x) { return f2d_exact(x.hi) + f2d_exact(x.lo); }

}  // namespace chx
