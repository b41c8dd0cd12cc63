// Host build of the double-float arithmetic of the CUDA path
// (paper_1303_4916_gb300/csrc/df64.cuh) for tests/test_df64_host.py (test
// infrastructure).  The device intrinsics it uses are IEEE-754 operations
// rounded to nearest without contraction; on the host they are the plain
// float operations and fmaf, compiled with -ffp-contract=off.  rsqrtf is an
// approximation on the device; here 1/sqrtf stands in (the df64 Newton step
// that follows it is what is under test).
#include <cmath>
#define __device__
#define __host__
#define __forceinline__ inline
static inline float __fadd_rn(float a, float b) { return a + b; }
static inline float __fsub_rn(float a, float b) { return a - b; }
static inline float __fmul_rn(float a, float b) { return a * b; }
static inline float __fmaf_rn(float a, float b, float c) { return std::fmaf(a, b, c); }
static inline float __double2float_rn(double x) { return (float)x; }
static inline float rsqrtf(float x) { return 1.0f / std::sqrt(x); }
#include "df64.cuh"

// each operand / result is a (hi, lo) pair of floats
extern "C" void df_add2(const float* a, const float* b, float* r) { const df64 v = df64(a[0], a[1]) + df64(b[0], b[1]); r[0] = v.hi; r[1] = v.lo; }
extern "C" void df_sub2(const float* a, const float* b, float* r) { const df64 v = df64(a[0], a[1]) - df64(b[0], b[1]); r[0] = v.hi; r[1] = v.lo; }
extern "C" void df_mul2(const float* a, const float* b, float* r) { const df64 v = df64(a[0], a[1]) * df64(b[0], b[1]); r[0] = v.hi; r[1] = v.lo; }
extern "C" void df_mulf2(const float* a, float b, float* r) { const df64 v = df_mulf(df64(a[0], a[1]), b); r[0] = v.hi; r[1] = v.lo; }
extern "C" void df_fma2(const float* a, const float* b, const float* c, float* r) {
  const df64 v = df_fma(df64(a[0], a[1]), df64(b[0], b[1]), df64(c[0], c[1])); r[0] = v.hi; r[1] = v.lo;
}
extern "C" void df_rsqrt2(const float* a, float* r) { const df64 v = rsqrt(df64(a[0], a[1])); r[0] = v.hi; r[1] = v.lo; }
extern "C" void df_from_double(double x, float* r) { const df64 v(x); r[0] = v.hi; r[1] = v.lo; }
