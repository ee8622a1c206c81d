// pff_df64.cuh -- double-word ("float-float") arithmetic on the FP32 pipe.
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2, about 48 bits of
// significand. The building blocks are the error-free transformations TwoSum (Knuth), Fast2Sum
// (Dekker, |a| >= |b|) and TwoProd via a fused multiply-add; the double-word operations follow
// the algorithms analysed by Joldes, Muller and Popescu (ACM TOMS 44, 2017): a product with the
// cross terms folded into the error term and a "sloppy" double-word addition whose error is
// bounded relative to |x| + |y|. Every primitive uses the _rn intrinsics so that the compiler
// cannot contract a product and a sum into one FMA, which would break the error-free transforms.
//
// On GB300 the FP64 pipe delivers 1/62 of the FP32 rate; a double-word multiply-add costs 15 FP32
// instructions, so kernels bound by FP64 arithmetic run several times faster in this form.
#pragma once
#include <cuda_runtime.h>

namespace pff {

struct df64 {
  float hi, lo;
  df64() = default;
  __host__ __device__ constexpr df64(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ constexpr explicit df64(int v) : hi((float)v), lo(0.f) {}
};

__host__ __device__ constexpr df64 df_make(float h, float l) { return df64(h, l); }
// Compile-time split of a double constant into a double-word pair.
__host__ __device__ constexpr df64 df_const(double d) { return df64((float)d, (float)(d - (double)(float)d)); }

// Error-free sum: s + e = a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float aa = __fsub_rn(s, bb);
  e = __fadd_rn(__fsub_rn(a, aa), __fsub_rn(b, bb));
}
// Error-free sum for |a| >= |b| (or a == 0).
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ df64 df_from(double d) {
  const float h = __double2float_rn(d);
  return df_make(h, __double2float_rn(d - (double)h));
}
__device__ __forceinline__ double df_to(df64 a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ df64 operator+(df64 x, df64 y) {
  float s, e;
  two_sum(x.hi, y.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(x.lo, y.lo));
  float zh, zl;
  fast_two_sum(s, e, zh, zl);
  return df_make(zh, zl);
}
__device__ __forceinline__ df64 operator-(df64 x) { return df_make(-x.hi, -x.lo); }
__device__ __forceinline__ df64 operator-(df64 x, df64 y) { return x + (-y); }
__device__ __forceinline__ df64 operator*(df64 x, df64 y) {
  const float ph = __fmul_rn(x.hi, y.hi);
  float pl = __fmaf_rn(x.hi, y.hi, -ph);
  pl = __fmaf_rn(x.hi, y.lo, pl);
  pl = __fmaf_rn(x.lo, y.hi, pl);
  float zh, zl;
  fast_two_sum(ph, pl, zh, zl);
  return df_make(zh, zl);
}
__device__ __forceinline__ df64& operator+=(df64& x, df64 y) {
  x = x + y;
  return x;
}

// x * y + c with one normalisation (15 FP32 instructions).
__device__ __forceinline__ df64 fmac(df64 x, df64 y, df64 c) {
  const float ph = __fmul_rn(x.hi, y.hi);
  float pl = __fmaf_rn(x.hi, y.hi, -ph);
  pl = __fmaf_rn(x.hi, y.lo, pl);
  pl = __fmaf_rn(x.lo, y.hi, pl);
  float s, e;
  two_sum(ph, c.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(pl, c.lo));
  float zh, zl;
  fast_two_sum(s, e, zh, zl);
  return df_make(zh, zl);
}
__device__ __forceinline__ double fmac(double x, double y, double c) { return fma(x, y, c); }
__device__ __forceinline__ float fmac(float x, float y, float c) { return fmaf(x, y, c); }

// Conversions between storage and compute types.
template <typename To, typename From>
__device__ __forceinline__ To cvt(From v) {
  return To(v);
}
template <>
__device__ __forceinline__ df64 cvt<df64, double>(double v) {
  return df_from(v);
}
template <>
__device__ __forceinline__ double cvt<double, df64>(df64 v) {
  return df_to(v);
}
// Constants in the compute type (double-word pairs split at compile time).
template <typename Real>
__host__ __device__ constexpr Real rconst(double v) {
  return Real(v);
}
template <>
__host__ __device__ constexpr df64 rconst<df64>(double v) {
  return df_const(v);
}

}  // namespace pff
