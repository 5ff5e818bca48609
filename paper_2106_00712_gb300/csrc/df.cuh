// Double-float ("FP32 pair") arithmetic for the compensated precision mode.
//
// A value is held as hi + lo with two floats, |lo| <= ulp(hi)/2, giving about 48 bits of
// significand on the FP32 pipes. Products and sums use error-free transformations:
// TwoProd by FMA (p = fl(a*b), e = fma(a, b, -p) exactly) and Knuth's TwoSum
// (s = fl(a+b), e = (a - (s - bb)) + (b - bb), bb = s - a) (Dekker 1971; Knuth, TAOCP
// vol. 2, 4.2.2). Every rounding step uses the _rn intrinsics so the compiler cannot
// contract or reassociate them.
#pragma once
#include <cuda_runtime.h>

namespace nmc {

struct __align__(8) df2 {
  float hi, lo;
};

__device__ __forceinline__ df2 df_zero() { return df2{0.f, 0.f}; }

__device__ __forceinline__ df2 df_from_double(double x) {
  const float hi = __double2float_rn(x);
  const float lo = __double2float_rn(x - (double)hi);
  return df2{hi, lo};
}

__device__ __forceinline__ double df_to_double(df2 a) { return (double)a.hi + (double)a.lo; }

// Fast2Sum renormalisation (requires |hi| >= |lo| up to a factor, true after the steps below)
__device__ __forceinline__ df2 df_norm(float hi, float lo) {
  const float s = __fadd_rn(hi, lo);
  const float e = __fsub_rn(lo, __fsub_rn(s, hi));
  return df2{s, e};
}

// acc += a * b, accumulator kept unnormalised (hi exact partial sum, lo running error)
__device__ __forceinline__ void df_fma_acc(df2& acc, df2 a, df2 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
  const float s = __fadd_rn(acc.hi, p);
  const float bb = __fsub_rn(s, acc.hi);
  const float t = __fadd_rn(__fsub_rn(acc.hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  acc.hi = s;
  acc.lo = __fadd_rn(acc.lo, __fadd_rn(t, e));
}

__device__ __forceinline__ df2 df_finish(df2 acc) { return df_norm(acc.hi, acc.lo); }

__device__ __forceinline__ df2 df_mul(df2 a, df2 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
  return df_norm(p, e);
}

__device__ __forceinline__ df2 df_add(df2 a, df2 b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  const float t = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  return df_norm(s, __fadd_rn(t, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ df2 df_neg(df2 a) { return df2{-a.hi, -a.lo}; }

__device__ __forceinline__ df2 df_abs(df2 a) { return a.hi < 0.f ? df_neg(a) : a; }

// 1/a: FP32 reciprocal, then one Newton step r + r (1 - a r) in double-float
// (doubles the correct bits, ~2^-44 relative).
__device__ __forceinline__ df2 df_rcp(df2 a) {
  const float r0 = __frcp_rn(a.hi);
  const df2 r{r0, 0.f};
  const df2 e = df_add(df2{1.f, 0.f}, df_neg(df_mul(a, r)));
  return df_add(r, df_mul(r, e));
}

}  // namespace nmc
