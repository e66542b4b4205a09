// Double-float ("df64") arithmetic: a value is the unevaluated sum hi + lo of
// two FP32 numbers with |lo| <= ulp(hi)/2, giving a 48-bit significand. Built
// from the error-free transformations of Dekker (1971) and Knuth (TAOCP vol. 2,
// sec. 4.2.2): TwoSum returns a + b exactly as s + e; TwoProd returns a * b
// exactly as p + e using one fused multiply-add. The adds below are the
// "sloppy" double-float adds of Dekker's paper (error ~2^-44 of the operands'
// magnitudes), which is the accuracy the solver needs for its
// FP64-accuracy products and updates.
#pragma once

#include <cuda_runtime.h>

namespace gsk {

struct df {
  float hi, lo;
};

__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return {s, e};
}
__device__ __forceinline__ df fast_two_sum(float a, float b) {   // requires |a| >= |b| or a == 0
  const float s = a + b;
  return {s, b - (s - a)};
}
__device__ __forceinline__ df two_prod(float a, float b) {
  const float p = a * b;
  return {p, fmaf(a, b, -p)};
}
__device__ __forceinline__ df df_from_double(double x) {
  const float h = (float)x;
  return {h, (float)(x - (double)h)};
}
__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ df df_from_float2(float2 v) { return {v.x, v.y}; }
__device__ __forceinline__ float2 df_to_float2(df a) { return make_float2(a.hi, a.lo); }

__device__ __forceinline__ df df_add(df a, df b) {
  const df s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}
__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }
__device__ __forceinline__ df df_mul(df a, df b) {
  df p = two_prod(a.hi, b.hi);
  p.lo = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo));
  return fast_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ df df_mul_f(df a, float b) {
  df p = two_prod(a.hi, b);
  p.lo = fmaf(a.lo, b, p.lo);
  return fast_two_sum(p.hi, p.lo);
}

// Accumulator of a sum of products a * x: hi carries the running sum of the
// rounded leading products (kept exact by TwoSum), lo collects every rounding
// error and the cross terms. Renormalised once, when the sum is read.
struct dfacc {
  float hi, lo;
};
__device__ __forceinline__ void acc_zero(dfacc& s) { s.hi = 0.f; s.lo = 0.f; }
// s += a * x with a, x double-float
__device__ __forceinline__ void acc_fma(dfacc& s, float2 a, float2 x) {
  const float p = a.x * x.x;
  const float e = fmaf(a.x, x.x, -p);
  const float t = s.hi + p;
  const float bb = t - s.hi;
  const float err = (s.hi - (t - bb)) + (p - bb);
  s.hi = t;
  s.lo += (err + e) + fmaf(a.x, x.y, a.y * x.x);
}
// s += a * x with a double-float, x single
__device__ __forceinline__ void acc_fma(dfacc& s, float2 a, float x) {
  const float p = a.x * x;
  const float e = fmaf(a.x, x, -p);
  const float t = s.hi + p;
  const float bb = t - s.hi;
  const float err = (s.hi - (t - bb)) + (p - bb);
  s.hi = t;
  s.lo = fmaf(a.y, x, s.lo + (err + e));
}
__device__ __forceinline__ df acc_value(const dfacc& s) { return two_sum(s.hi, s.lo); }

}  // namespace gsk
