// Double-float arithmetic: a value is the unevaluated sum hi + lo of two
// FP32 numbers (|lo| <= ulp(hi)/2), about 48 significant bits.  On this GPU
// an FP64 instruction costs about 64 cycles of latency and issues at ~1/64
// of the FP32 rate, so the latency-bound parts of the IB solve (vector
// updates, dot products, scalar recurrences) run in this format on the FP32
// pipes instead.  The building blocks are the published error-free
// transformations: TwoSum (Knuth, TAOCP Vol. 2, Sec. 4.2.2), FastTwoSum
// (Dekker 1971), TwoProduct through a fused multiply-add, and compensated
// summation in the style of Ogita, Rump and Oishi (2005).  Every operation
// uses explicitly rounded intrinsics (__fadd_rn, __fmul_rn, fmaf) so that
// compiler contraction cannot change an error term.
#pragma once

#include <cuda_runtime.h>

namespace ibl {

struct __align__(8) df {
  float hi, lo;
};

__device__ __forceinline__ df df_make(float hi, float lo) {
  df r;
  r.hi = hi;
  r.lo = lo;
  return r;
}

// s + e = a + b exactly (any a, b).
__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return df_make(s, e);
}

// s + e = a + b exactly when |a| >= |b| (or a == 0).
__device__ __forceinline__ df fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float e = __fsub_rn(b, __fsub_rn(s, a));
  return df_make(s, e);
}

__device__ __forceinline__ df df_from_float(float a) { return df_make(a, 0.f); }

// Conversions at the boundary of the double-float region (FP64 work, used
// once per element and solve).
__device__ __forceinline__ df df_from_double(double d) {
  const float hi = __double2float_rn(d);
  const float lo = __double2float_rn(d - (double)hi);
  return df_make(hi, lo);
}
__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ df df_neg(df a) { return df_make(-a.hi, -a.lo); }

// a > b for normalised double-floats (hi carries the rounded value).
__device__ __forceinline__ bool df_greater(df a, df b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }

// a + b with the accurate (IEEE-style) double-float addition.  Commutative:
// both error terms are exact, so a + b and b + a give the same bits.
__device__ __forceinline__ df df_add(df a, df b) {
  df s = two_sum(a.hi, b.hi);
  const df t = two_sum(a.lo, b.lo);
  s.lo = __fadd_rn(s.lo, t.hi);
  s = fast_two_sum(s.hi, s.lo);
  s.lo = __fadd_rn(s.lo, t.lo);
  return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

// a * b (double-float times double-float).
__device__ __forceinline__ df df_mul(df a, df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}

// a * b (double-float times float).
__device__ __forceinline__ df df_mul_f(df a, float b) {
  const float p = __fmul_rn(a.hi, b);
  float e = fmaf(a.hi, b, -p);
  e = fmaf(a.lo, b, e);
  return fast_two_sum(p, e);
}

// a / b: three FP32 quotient digits with exact residuals.
__device__ __forceinline__ df df_div(df a, df b) {
  const float q1 = __fdiv_rn(a.hi, b.hi);
  df r = df_sub(a, df_mul_f(b, q1));
  const float q2 = __fdiv_rn(r.hi, b.hi);
  r = df_sub(r, df_mul_f(b, q2));
  const float q3 = __fdiv_rn(r.hi, b.hi);
  const df q = fast_two_sum(q1, q2);
  return df_add(q, df_from_float(q3));
}

// Compensated accumulator: s holds the FP32 running sum, c the accumulated
// rounding errors of the additions and the low parts of the terms; the
// value is s + c, rounded to a double-float by acc_value.
struct dfacc {
  float s, c;
};
__device__ __forceinline__ dfacc acc_zero() {
  dfacc a;
  a.s = 0.f;
  a.c = 0.f;
  return a;
}
// a += x * y with x double-float and y float (TwoProduct of the high part).
__device__ __forceinline__ void acc_fma_f(dfacc& a, df x, float y) {
  const float p = __fmul_rn(x.hi, y);
  const float e = fmaf(x.lo, y, fmaf(x.hi, y, -p));
  const df t = two_sum(a.s, p);
  a.s = t.hi;
  a.c = __fadd_rn(a.c, __fadd_rn(t.lo, e));
}
// a += x * y, both double-float.
__device__ __forceinline__ void acc_fma(dfacc& a, df x, df y) {
  const float p = __fmul_rn(x.hi, y.hi);
  const float e = fmaf(x.lo, y.hi, fmaf(x.hi, y.lo, fmaf(x.hi, y.hi, -p)));
  const df t = two_sum(a.s, p);
  a.s = t.hi;
  a.c = __fadd_rn(a.c, __fadd_rn(t.lo, e));
}
// a += x * y, both float: the product's rounding error enters c exactly.
__device__ __forceinline__ void acc_fma_ff(dfacc& a, float x, float y) {
  const float p = __fmul_rn(x, y);
  const float e = fmaf(x, y, -p);
  const df t = two_sum(a.s, p);
  a.s = t.hi;
  a.c = __fadd_rn(a.c, __fadd_rn(t.lo, e));
}
__device__ __forceinline__ df acc_value(dfacc a) { return fast_two_sum(a.s, a.c); }

// Butterfly sum over groups of `width` lanes in a fixed order (every lane of
// a group ends with the same total).
__device__ __forceinline__ df df_warp_sum(df v, int width = 32) {
  for (int o = width >> 1; o > 0; o >>= 1) {
    const df w = df_make(__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o));
    v = df_add(v, w);
  }
  return v;
}

}  // namespace ibl
