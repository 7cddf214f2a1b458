// Double-float (unevaluated FP32 pair hi + lo) arithmetic for the few values
// whose FP32 rounding would swamp a dd residual: distances, travel times and
// their differences.  Error-free transforms: Knuth's TwoSum, Dekker's
// Fast2Sum, and the FMA form of TwoProduct.
#pragma once
#include <cuda_runtime.h>

namespace spider {

struct df32 {
  float hi, lo;
};

__device__ __forceinline__ df32 df_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

__device__ __forceinline__ df32 df_fast_two_sum(float a, float b) {  // |a| >= |b|
  float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ df32 df_two_prod(float a, float b) {
  float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ df32 df_add(df32 a, df32 b) {
  df32 s = df_two_sum(a.hi, b.hi);
  float lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return df_fast_two_sum(s.hi, lo);
}

__device__ __forceinline__ df32 df_add_f(df32 a, float b) {
  df32 s = df_two_sum(a.hi, b);
  return df_fast_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}

__device__ __forceinline__ df32 df_mul(df32 a, df32 b) {
  df32 p = df_two_prod(a.hi, b.hi);
  float lo = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
  return df_fast_two_sum(p.hi, lo);
}

__device__ __forceinline__ df32 df_mul_f(df32 a, float b) {
  df32 p = df_two_prod(a.hi, b);
  return df_fast_two_sum(p.hi, __fmaf_rn(a.lo, b, p.lo));
}

__device__ __forceinline__ df32 df_sqr(df32 a) {
  df32 p = df_two_prod(a.hi, a.hi);
  float lo = __fmaf_rn(__fmul_rn(2.0f, a.hi), a.lo, p.lo);
  return df_fast_two_sum(p.hi, lo);
}

// sqrt by one Newton correction of the FP32 root: s + (a - s^2) / (2 s)
__device__ __forceinline__ df32 df_sqrt(df32 a) {
  float s = sqrtf(a.hi);
  df32 s2 = df_two_prod(s, s);
  float resid = __fadd_rn(__fsub_rn(__fsub_rn(a.hi, s2.hi), s2.lo), a.lo);
  return df_fast_two_sum(s, __fdiv_rn(resid, __fmul_rn(2.0f, s)));
}

// difference of two coordinates each given as (hi, lo) plus a small offset on the first
__device__ __forceinline__ df32 df_coord_diff(float ahi, float alo, float aoff, float bhi, float blo) {
  df32 d = df_two_sum(ahi, -bhi);
  return df_add_f(d, __fadd_rn(__fsub_rn(alo, blo), aoff));
}

}  // namespace spider
