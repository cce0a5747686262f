// Float-float ("double-single") arithmetic: a value is the unevaluated sum hi + lo of
// two floats with |lo| <= ulp(hi)/2, about 48 significant bits. Built from the
// error-free transformations of Knuth (TwoSum), Dekker (Fast2Sum) and the
// FMA-based exact product, so every operation runs on the FP32 pipes. Used for the
// refinement residual, where a GPU with a low double-precision rate would otherwise
// spend most of its time.
#pragma once
#include <cuda_runtime.h>

namespace mlmc {

struct DF {
  float hi, lo;
};

__device__ __forceinline__ DF df(float a) { return DF{a, 0.f}; }

// Exact double -> float-float split (two conversions and one subtraction).
__device__ __forceinline__ DF df_from_double(double a) {
  const float hi = __double2float_rn(a);
  return DF{hi, __double2float_rn(a - (double)hi)};
}

__device__ __forceinline__ double df_to_double(DF a) { return (double)a.hi + (double)a.lo; }

// Knuth TwoSum: s + e = a + b exactly.
__device__ __forceinline__ DF two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return DF{s, e};
}

// Dekker Fast2Sum, |a| >= |b|: s + e = a + b exactly.
__device__ __forceinline__ DF fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return DF{s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ DF operator+(DF a, DF b) {
  DF s = two_sum(a.hi, b.hi);
  const DF t = two_sum(a.lo, b.lo);
  s.lo = __fadd_rn(s.lo, t.hi);
  s = fast_two_sum(s.hi, s.lo);
  s.lo = __fadd_rn(s.lo, t.lo);
  return fast_two_sum(s.hi, s.lo);
}

// The shorter float-float sum: the heads by TwoSum, the tails added once. Its error is
// about 2^-47 (|a| + |b|) rather than 2^-47 |a + b|: as good as operator+ where the
// operands are no larger than the scale the result is needed at, not where two large
// values cancel to a small one.
__device__ __forceinline__ DF df_add_short(DF a, DF b) {
  const DF s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ DF df_sub_short(DF a, DF b) { return df_add_short(a, DF{-b.hi, -b.lo}); }

__device__ __forceinline__ DF operator-(DF a) { return DF{-a.hi, -a.lo}; }
__device__ __forceinline__ DF operator-(DF a, DF b) { return a + (-b); }

// float-float times float: exact product of the heads by FMA, plus the tail term.
__device__ __forceinline__ DF operator*(DF a, float b) {
  const float p = __fmul_rn(a.hi, b);
  const float e = __fmaf_rn(a.hi, b, -p);
  return fast_two_sum(p, __fmaf_rn(a.lo, b, e));
}

__device__ __forceinline__ DF operator*(float b, DF a) { return a * b; }

// acc += a * b for float-float a and b: the exact product of the heads by FMA, the two
// cross terms, then TwoSum into the accumulator.
__device__ __forceinline__ void df_fma(DF& acc, DF a, DF b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const DF s = two_sum(acc.hi, p);
  acc = fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(e, acc.lo)));
}

__device__ __forceinline__ DF shfl_down_df(DF a, int d) {
  return DF{__shfl_down_sync(0xffffffffu, a.hi, d), __shfl_down_sync(0xffffffffu, a.lo, d)};
}
__device__ __forceinline__ DF shfl_up_df(DF a, int d) {
  return DF{__shfl_up_sync(0xffffffffu, a.hi, d), __shfl_up_sync(0xffffffffu, a.lo, d)};
}

}  // namespace mlmc
