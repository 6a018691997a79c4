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
__device__ __forceinline__ ff d2ff_general(double x) {
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

// The same split by a short path, exact for 2^-74 <= |x| < 2^128 (both parts
// are then normal floats): hi's exponent and top 23 significand bits are one
// funnel shift of the double's two words, rebiased by one subtraction (the
// exponent field is taken mod 2^9, and e - 896 lies in [53, 254] there, so the
// wrap-around restores it); lo is the low 29 significand bits converted and
// scaled by 2^(e - 1075).  No branch: `bad` is set when x is outside that
// range, and the caller then redoes its batch with d2ff_general (so a batch's
// loads are all issued before any test of their values).  Where it applies the
// bits equal d2ff_general's, zero lo included.
__device__ __forceinline__ ff d2ff_fast(double x, bool& bad) {
  const uint32_t w1 = (uint32_t)__double2hiint(x), w0 = (uint32_t)__double2loint(x);
  const uint32_t e = (w1 >> 20) & 0x7ffu;
  bad = bad || e - 949u >= 202u;
  const uint32_t sgn = w1 & 0x80000000u;
  const float hi = __uint_as_float((__funnelshift_l(w0, w1, 3) - 0xC0000000u) | sgn);  // 896 << 23, mod 2^32
  const uint32_t r = w0 & 0x1FFFFFFFu;
  const float lo = __uint2float_rn(r) * __uint_as_float((e - 948u) << 23);
  return ff{hi, r ? __uint_as_float(__float_as_uint(lo) | sgn) : 0.f};
}

__device__ __forceinline__ ff d2ff(double x) { return d2ff_general(x); }

// Exact float -> double by bit manipulation (denormal floats flush to zero).
// Normal floats take the short path: exponent rebiased by 896 in the high word,
// the significand's low 3 bits at the top of the low word.
__device__ __forceinline__ double f2d_exact(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t a = u & 0x7fffffffu;
  if (a - 0x00800000u < 0x7f000000u)
    return __hiloint2double((int)(((a >> 3) + (896u << 20)) | (u & 0x80000000u)), (int)(u << 29));
  const uint32_t e = (u >> 23) & 0xff;
  const uint64_t sgn = (uint64_t)(u >> 31) << 63;
  if (e == 0) return __longlong_as_double((long long)sgn);
  if (e == 255) return __longlong_as_double((long long)(sgn | 0x7ff0000000000000ull | ((uint64_t)(u & 0x7fffff) << 29)));
  return __longlong_as_double((long long)(sgn | ((uint64_t)(e + 896) << 52) | ((uint64_t)(u & 0x7fffff) << 29)));
}

// ff -> FP64: both parts convert exactly; one FP64 add rounds the sum.
__device__ __forceinline__ double ff2d(ff x) { return f2d_exact(x.hi) + f2d_exact(x.lo); }

}  // namespace chx

// ---------------------------------------------------------------------------
// The same operations on two independent values at once, with the packed FP32
// instructions of sm_100 and later (__fadd2_rn, __fmul2_rn, __ffma2_rn): one
// instruction rounds each lane as its scalar form would, so a pair's results
// are bit-identical to two scalar calls, in half the instructions.
namespace chx {

struct ff2 {
  float2 hi, lo;
};

__device__ __forceinline__ float2 f2neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b, rounded once (the product with -1 is exact)
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }

__device__ __forceinline__ ff2 fast_two_sum2(float2 a, float2 b) {
  const float2 s = f2add(a, b);
  return ff2{s, f2sub(b, f2sub(s, a))};
}

__device__ __forceinline__ ff2 two_sum2(float2 a, float2 b) {
  const float2 s = f2add(a, b);
  const float2 bb = f2sub(s, a);
  return ff2{s, f2add(f2sub(a, f2sub(s, bb)), f2sub(b, bb))};
}

__device__ __forceinline__ ff2 two_prod2(float2 a, float2 b) {
  const float2 p = __fmul2_rn(a, b);
  return ff2{p, __ffma2_rn(a, b, f2neg(p))};
}

__device__ __forceinline__ ff2 ff2_add(ff2 x, ff2 y) {
  const ff2 s = two_sum2(x.hi, y.hi);
  return fast_two_sum2(s.hi, f2add(s.lo, f2add(x.lo, y.lo)));
}

__device__ __forceinline__ ff2 ff2_sub(ff2 x, ff2 y) { return ff2_add(x, ff2{f2neg(y.hi), f2neg(y.lo)}); }

__device__ __forceinline__ ff2 ff2_add_f(ff2 x, float2 y) {
  const ff2 s = two_sum2(x.hi, y);
  return fast_two_sum2(s.hi, f2add(s.lo, x.lo));
}

__device__ __forceinline__ ff2 ff2_mul(ff2 x, ff2 y) {
  const ff2 p = two_prod2(x.hi, y.hi);
  float2 e = __ffma2_rn(x.hi, y.lo, p.lo);
  e = __ffma2_rn(x.lo, y.hi, e);
  return fast_two_sum2(p.hi, e);
}

__device__ __forceinline__ ff2 ff2_scale2(ff2 x, float p2) {
  const float2 s = make_float2(p2, p2);
  return ff2{__fmul2_rn(x.hi, s), __fmul2_rn(x.lo, s)};
}

// pack / unpack two scalar double-float values
__device__ __forceinline__ ff2 ff2_pack(ff a, ff b) { return ff2{make_float2(a.hi, b.hi), make_float2(a.lo, b.lo)}; }
__device__ __forceinline__ ff ff2_first(ff2 v) { return ff{v.hi.x, v.lo.x}; }
__device__ __forceinline__ ff ff2_second(ff2 v) { return ff{v.hi.y, v.lo.y}; }
__device__ __forceinline__ ff2 ff2_splat(ff a) { return ff2{make_float2(a.hi, a.hi), make_float2(a.lo, a.lo)}; }

}  // namespace chx
