// df64.cuh -- double-float ("df64") arithmetic on the FP32 pipe.
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2,
// a 48-bit significand (unit roundoff 2^-48 ~ 3.6e-15) over the float
// exponent range.  GB300 runs FP32 at 61x its FP64 rate (76.5 vs 1.25
// TFLOP/s measured), so recurrences that need about 1e-14 relative accuracy
// run faster in df64 than in native FP64.
//
// The operations are the classic error-free transformations (Dekker 1971,
// Knuth TAOCP vol. 2): two-sum, quick-two-sum and the FMA-based two-product.
// They are written with the __fadd_rn / __fmul_rn intrinsics, which the
// compiler never contracts into FMAs, so the error terms stay exact.
#pragma once
#include <cuda_runtime.h>

struct df64 {
  float hi, lo;
  df64() = default;
  __host__ __device__ constexpr df64(float h, float l) : hi(h), lo(l) {}
  __device__ __forceinline__ explicit df64(int k) : hi((float)k), lo(0.f) {}
  // from double: hi = rn(x), lo = rn(x - hi) (uses the FP64 unit: setup only)
  __device__ __forceinline__ explicit df64(double x) {
    hi = __double2float_rn(x);
    lo = __double2float_rn(x - (double)hi);
  }
  __device__ __forceinline__ explicit operator double() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ df64 df_quick_two_sum(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  const float e = __fsub_rn(b, __fsub_rn(s, a));
  return df64(s, e);
}

__device__ __forceinline__ df64 operator+(df64 a, df64 b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  return df_quick_two_sum(s, e);
}

__device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.hi, -a.lo); }
__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }

__device__ __forceinline__ df64 operator*(df64 a, df64 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_quick_two_sum(p, e);
}

// df64 times a float
__device__ __forceinline__ df64 df_mulf(df64 a, float b) {
  const float p = __fmul_rn(a.hi, b);
  float e = __fmaf_rn(a.hi, b, -p);
  e = __fmaf_rn(a.lo, b, e);
  return df_quick_two_sum(p, e);
}

// a*b + c with one final normalisation (the product's error term joins the
// two-sum of the addition)
__device__ __forceinline__ df64 df_fma(df64 a, df64 b, df64 c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const float s = __fadd_rn(p, c.hi);
  const float bb = __fsub_rn(s, p);
  float err = __fadd_rn(__fsub_rn(p, __fsub_rn(s, bb)), __fsub_rn(c.hi, bb));
  err = __fadd_rn(err, __fadd_rn(e, c.lo));
  return df_quick_two_sum(s, err);
}

// a * b + c, the fused step the generated recurrences call for every
// arithmetic type (FP64 and FP32 have theirs in the generated header)
__device__ __forceinline__ df64 fmac(df64 a, df64 b, df64 c) { return df_fma(a, b, c); }

// exact scaling by a power of two
__device__ __forceinline__ df64 df_scale2(df64 a, float pow2) { return df64(a.hi * pow2, a.lo * pow2); }

__device__ __forceinline__ df64& operator+=(df64& a, df64 b) {
  a = a + b;
  return a;
}

// 1/sqrt(a): float estimate refined by one Newton step in df64,
// y1 = y0 + y0 (1 - a y0^2) / 2 (relative error ~ 2^-46).
__device__ __forceinline__ df64 rsqrt(df64 a) {
  const float y = rsqrtf(a.hi);
  const float y2 = __fmul_rn(y, y);
  const float y2e = __fmaf_rn(y, y, -y2);  // y^2 = y2 + y2e exactly
  const df64 ay2 = a * df64(y2, y2e);
  const df64 r = df64(1.0f, 0.0f) - ay2;  // small
  const float corr = __fmul_rn(__fmul_rn(0.5f, y), r.hi);
  return df_quick_two_sum(y, corr);
}
