// eri.cuh -- per-class ERI kernels with the fused J/K contraction.
//
// One thread evaluates one contracted shell quartet (ab|cd) of Eq. 5; the
// 32 lanes of a warp share the bra pair (ab) and take 32 consecutive kets
// (cd) from the Schwarz-sorted ket list.  Per primitive quartet the thread
// evaluates the Boys function F_m(T), m = 0..L, and the Obara-Saika VRR
// (generated per class), accumulating [e0|f0]; after the primitive loop the
// HRR gives the Cartesian block, which is digested straight into J and K
// (the J/K equation of Sec. "Technical details").
//
// Digestion of one unique quartet with block I_abcd and degeneracy weight
// w = 1 / |stabiliser| (1/2 for each of A==B, C==D, (AB)==(CD)):
//   J'_ab += w sum_cd I D_cd          J'_cd += w sum_ab I D_ab
//   K'_ac += w sum_bd I D_bd          K'_ad += w sum_bc I D_bc
//   K'_bc += w sum_ad I D_ad          K'_bd += w sum_ac I D_ac
// and at the end J = 2 (J' + J'^T), K = K' + K'^T.  This sums the block
// over the full 8-member orbit of (ab|cd) under the permutational symmetry
// of Eq. 5 for a symmetric D.  J'_ab is reduced over the warp with
// shuffles before one FP64 atomic per element; the other five go out as
// FP64 atomics per lane.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "df64.cuh"
#include "eri_classes.cuh"
#include "hf_device.h"
#include "rys.cuh"

namespace hfk {

// ------------------------------------------------------------- Boys function
// For T < BOYS_TMAX, with T_i the nearest grid point and x = T_i - T
// (|x| <= BOYS_H/2): F_m(T) = sum_k F_{m+k}(T_i) x^k / k!  (dF_m/dT =
// -F_{m+1}) by Horner on the pre-divided coefficients of slice m, 8 terms
// (truncation below 1e-15 relative).  For L <= 1 every order is taken this
// way; for L >= 2 only F_L, then exp(-T) = exp(-T_i) e^x the same way and
// the downward recursion F_m = (2T F_{m+1} + exp(-T)) / (2m+1).  For
// T >= BOYS_TMAX: F_0 = sqrt(pi/T)/2 and F_{m+1} = (2m+1) F_m / (2T); the
// neglected exp(-T) terms are below 1e-26.
// The row index is rounded with the 1.5 * 2^52 shifter (no conversions):
// the low word of T/h + 1.5 * 2^52 is round(T/h).
#define HF_ROUND_SHIFTER 6755399441055744.0

__device__ __forceinline__ double boys_horner64(const double* __restrict__ c, double x) {
  const double2* c2 = reinterpret_cast<const double2*>(c);
  const double2 a = __ldg(c2), b = __ldg(c2 + 1), d = __ldg(c2 + 2), e = __ldg(c2 + 3);
  double f = e.y;
  f = fma(f, x, e.x);
  f = fma(f, x, d.y);
  f = fma(f, x, d.x);
  f = fma(f, x, b.y);
  f = fma(f, x, b.x);
  f = fma(f, x, a.y);
  return fma(f, x, a.x);
}

template <int L>
__device__ __forceinline__ void boys64(double T, const double* __restrict__ tab, double* F) {
  if (T < BOYS_TMAX) {
    const double y = fma(T, 1.0 / BOYS_H, HF_ROUND_SHIFTER);
    const int i = __double2loint(y);
    const double x = fma(y - HF_ROUND_SHIFTER, BOYS_H, -T);
    if (L <= 1) {
#pragma unroll
      for (int m = 0; m <= L; ++m) F[m] = boys_horner64(tab + ((size_t)m * BOYS_NGRID + i) * BOYS64_ROW, x);
    } else {
      const double* __restrict__ r = tab + ((size_t)L * BOYS_NGRID + i) * BOYS64_ROW;
      F[L] = boys_horner64(r, x);
      const double e = boys_horner64(r + BOYS64_TERMS, x);
      const double t2 = 2.0 * T;
#pragma unroll
      for (int m = L - 1; m >= 0; --m) F[m] = fma(t2, F[m + 1], e) * (1.0 / (2 * m + 1));
    }
  } else {
    const double rt = rsqrt(T);
    const double o2t = 0.5 * rt * rt;
    F[0] = 0.88622692545275801365 * rt;  // sqrt(pi)/2
#pragma unroll
    for (int m = 0; m < L; ++m) F[m + 1] = F[m] * ((2 * m + 1) * o2t);
  }
}

// FP32 evaluation of the same expansion, 5 terms (truncation below 3e-9
// relative), for the reduced-precision quartets when requested.
__device__ __forceinline__ float boys_horner32(const float* __restrict__ c, float x) {
  float f = __ldg(c + 4);
  f = fmaf(f, x, __ldg(c + 3));
  f = fmaf(f, x, __ldg(c + 2));
  f = fmaf(f, x, __ldg(c + 1));
  return fmaf(f, x, __ldg(c));
}

template <int L>
__device__ __forceinline__ void boys32(float T, const float* __restrict__ tab, float* F) {
  if (T < (float)BOYS_TMAX) {
    const int i = __float2int_rn(T * (float)(1.0 / BOYS_H));
    const float x = (float)i * (float)BOYS_H - T;
    if (L <= 1) {
#pragma unroll
      for (int m = 0; m <= L; ++m) F[m] = boys_horner32(tab + ((size_t)m * BOYS_NGRID + i) * BOYS32_ROW, x);
    } else {
      const float* __restrict__ r = tab + ((size_t)L * BOYS_NGRID + i) * BOYS32_ROW;
      F[L] = boys_horner32(r, x);
      const float e = boys_horner32(r + BOYS32_TERMS, x);
      const float t2 = 2.0f * T;
#pragma unroll
      for (int m = L - 1; m >= 0; --m) F[m] = fmaf(t2, F[m + 1], e) * (1.0f / (2 * m + 1));
    }
  } else {
    const float rt = rsqrtf(T);
    const float o2t = 0.5f * rt * rt;
    F[0] = 0.88622692545275801365f * rt;
#pragma unroll
    for (int m = 0; m < L; ++m) F[m + 1] = F[m] * ((2 * m + 1) * o2t);
  }
}

// ------------------------------------------------------------- primitive pairs
template <typename R>
struct Prim {
  R p, o2p, P[3], PA[3], K;
};

__device__ __forceinline__ void load_prim(const double* __restrict__ base, int idx, Prim<double>& q) {
  const double2* s = reinterpret_cast<const double2*>(base + (size_t)idx * PRIM64_STRIDE);
  const double2 a = __ldg(s), b = __ldg(s + 1), c = __ldg(s + 2), d = __ldg(s + 3), e = __ldg(s + 4);
  q.p = a.x; q.o2p = a.y; q.P[0] = b.x; q.P[1] = b.y; q.P[2] = c.x;
  q.PA[0] = c.y; q.PA[1] = d.x; q.PA[2] = d.y; q.K = e.x;
}

__device__ __forceinline__ void load_prim(const float* __restrict__ base, int idx, Prim<float>& q) {
  const float4* s = reinterpret_cast<const float4*>(base + (size_t)idx * PRIM32_STRIDE);
  const float4 a = __ldg(s), b = __ldg(s + 1), c = __ldg(s + 2);
  q.p = a.x; q.o2p = a.y; q.P[0] = a.z; q.P[1] = a.w; q.P[2] = b.x;
  q.PA[0] = b.y; q.PA[1] = b.z; q.PA[2] = b.w; q.K = c.x;
}

template <typename R> struct PrimBase;
template <> struct PrimBase<double> { static __device__ __forceinline__ const double* get(const PairSet& s) { return s.prim64; } };
template <> struct PrimBase<float> { static __device__ __forceinline__ const float* get(const PairSet& s) { return s.prim32; } };

template <int L, typename R>
struct BoysSel {
  static __device__ __forceinline__ void eval(R T, const KernelCommon& kc, R* F);
};
template <int L>
struct BoysSel<L, double> {
  static __device__ __forceinline__ void eval(double T, const KernelCommon& kc, double* F) {
    boys64<L>(T, kc.boys64, F);
  }
};
template <int L>
__device__ __forceinline__ void boys_df(df64 T, const float* __restrict__ tab, df64* F);

template <int L>
struct BoysSel<L, float> {
  // Reduced-precision quartets: F_m in FP64 (table + downward recursion),
  // rounded to FP32 for the recurrences; in df64 (same recursion, 48-bit
  // significand) in the df64 tier; in FP32 when boys_fp32 is set.
  static __device__ __forceinline__ void eval(float T, const KernelCommon& kc, float* F) {
    if (kc.boys_fp32) {
      boys32<L>(T, kc.boys32, F);
    } else if (kc.boys_df) {
      df64 Fd[L + 1];
      boys_df<L>(df64(T, 0.0f), kc.boysdf, Fd);
#pragma unroll
      for (int m = 0; m <= L; ++m) F[m] = __fadd_rn(Fd[m].hi, Fd[m].lo);
    } else {
      double Fd[L + 1];
      boys64<L>((double)T, kc.boys64, Fd);
#pragma unroll
      for (int m = 0; m <= L; ++m) F[m] = (float)Fd[m];
    }
  }
};

// Contracted block of one shell quartet: loops over the significant
// primitive pairs of bra and ket.  nb/nk are the primitive-pair counts
// (0 for an inactive lane).
template <class C, typename R>
__device__ __forceinline__ void contracted_vrr(const PairSet& ps, const KernelCommon& kc, int b0, int nb,
                                               int k0, int nk, R* acc) {
  const auto* base = PrimBase<R>::get(ps);
#pragma unroll
  for (int x = 0; x < C::NE * C::NF; ++x) acc[x] = (R)0;
  // ket primitives outer (a different record per lane, loaded once each),
  // bra primitives inner (the same record for the whole warp)
  for (int ik = 0; ik < nk; ++ik) {
    Prim<R> c;
    load_prim(base, k0 + ik, c);
    for (int ib = 0; ib < nb; ++ib) {
      Prim<R> a;
      load_prim(base, b0 + ib, a);
      const R pq = a.p + c.p;
      const R rs = (R)rsqrt(pq);
      const R inv = rs * rs;
      const R rp = c.p * inv;  // rho / zeta
      const R rq = a.p * inv;  // rho / eta
      R PQ[3], WP[3], WQ[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        PQ[i] = a.P[i] - c.P[i];
        WP[i] = -rp * PQ[i];
        WQ[i] = rq * PQ[i];
      }
      const R T = a.p * rp * (PQ[0] * PQ[0] + PQ[1] * PQ[1] + PQ[2] * PQ[2]);
      R B[C::L + 1];
      BoysSel<C::L, R>::eval(T, kc, B);
      const R pref = a.K * c.K * rs;
#pragma unroll
      for (int m = 0; m <= C::L; ++m) B[m] *= pref;
      C::template vrr<R>(acc, B, a.PA, WP, c.PA, WQ, a.o2p, c.o2p, (R)0.5 * inv, rp, rq);
    }
  }
}

// ------------------------------------------------------------- df64 path
// Boys in df64: grid T_i = i/16 (exact in FP32), x = T_i - T exact as a
// two-term sum (|x| <= 1/32).  F_L(T) = sum_{k<8} F_{L+k}(T_i) x^k/k! by
// Horner on the row's coefficients, the terms k >= 5 (below 2^-30 of the
// sum) in FP32 and k <= 4 in df64.  For L >= 1 also exp(-T) =
// exp(-T_i) e^x, with e^x = sum_{k<8} x^k/k! (truncation below 2^-55) by
// Horner on constant coefficients, then the downward recursion in df64.
// The row (16 floats, 64 bytes) comes in two 256-bit loads: per lane two
// 32-byte sectors instead of one 16-byte load per coefficient pair.
// T >= BOYS_TMAX: F_0 = sqrt(pi)/2 T^{-1/2}, F_{m+1} = (2m+1)/(2T) F_m.
struct BoysRowDf {
  float v[16];
};

__device__ __forceinline__ void ldg256(const float* __restrict__ p, float* v) {
  asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
      : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
      : "l"(p));
}

__device__ __forceinline__ BoysRowDf load_boys_row_df(const float* __restrict__ r) {
  BoysRowDf q;
  ldg256(r, q.v);
  ldg256(r + 8, q.v + 8);
  return q;
}

__device__ __forceinline__ df64 boys_horner_df(const BoysRowDf& q, df64 x) {
  float g = __fmaf_rn(q.v[12], x.hi, q.v[11]);  // c7 x + c6
  g = __fmaf_rn(g, x.hi, q.v[10]);              // + c5
  df64 f = df64(q.v[8], q.v[9]) + df_mulf(x, g);
  f = df_fma(x, f, df64(q.v[6], q.v[7]));
  f = df_fma(x, f, df64(q.v[4], q.v[5]));
  f = df_fma(x, f, df64(q.v[2], q.v[3]));
  return df_fma(x, f, df64(q.v[0], q.v[1]));
}

// (hi, lo) of a double constant
__device__ __forceinline__ constexpr df64 df_const(double v) { return df64((float)v, (float)(v - (double)(float)v)); }

// e^x for |x| <= 1/32: terms k = 5..7 in FP32, k <= 4 in df64
__device__ __forceinline__ df64 df_exp_small(df64 x) {
  float g = __fmaf_rn(1.0f / 5040.0f, x.hi, 1.0f / 720.0f);
  g = __fmaf_rn(g, x.hi, 1.0f / 120.0f);
  df64 f = df_const(1.0 / 24.0) + df_mulf(x, g);
  f = df_fma(x, f, df_const(1.0 / 6.0));
  f = df_fma(x, f, df64(0.5f, 0.0f));
  f = df_fma(x, f, df64(1.0f, 0.0f));
  return df_fma(x, f, df64(1.0f, 0.0f));
}

// (hi, lo) of 1/(2m+1), m = 0..7
__device__ __forceinline__ df64 df_inv_odd(int m) {
  constexpr double v[8] = {1.0, 1.0 / 3, 1.0 / 5, 1.0 / 7, 1.0 / 9, 1.0 / 11, 1.0 / 13, 1.0 / 15};
  const float h = (float)v[m];
  return df64(h, (float)(v[m] - (double)h));
}

template <int L>
__device__ __forceinline__ void boys_df(df64 T, const float* __restrict__ tab, df64* F) {
  if (T.hi < (float)BOYS_TMAX) {
    const int i = __float2int_rn(T.hi * BOYSDF_INV_H);
    const float xh = __fsub_rn((float)i * (1.0f / BOYSDF_INV_H), T.hi);  // exact (Sterbenz)
    const df64 x = df64(xh, 0.0f) + df64(-T.lo, 0.0f);
    const BoysRowDf q = load_boys_row_df(tab + ((size_t)L * BOYSDF_NGRID + i) * BOYSDF_ROW);
    F[L] = boys_horner_df(q, x);
    if (L > 0) {
      const df64 e = df64(q.v[14], q.v[15]) * df_exp_small(x);
      const df64 t2 = df_scale2(T, 2.0f);
#pragma unroll
      for (int m = L - 1; m >= 0; --m) F[m] = (t2 * F[m + 1] + e) * df_inv_odd(m);
    }
  } else {
    const df64 rt = rsqrt(T);
    const df64 o2t = df_scale2(rt * rt, 0.5f);
    constexpr double kHalfSqrtPi = 0.88622692545275801365;
    F[0] = rt * df64((float)kHalfSqrtPi, (float)(kHalfSqrtPi - (double)(float)kHalfSqrtPi));
#pragma unroll
    for (int m = 0; m < L; ++m) F[m + 1] = df_mulf(F[m] * o2t, (float)(2 * m + 1));
  }
}

__device__ __forceinline__ void load_prim_df(const float* __restrict__ base, int idx, Prim<df64>& q) {
  const float4* s = reinterpret_cast<const float4*>(base + (size_t)idx * PRIMDF_STRIDE);
  const float4 a = __ldg(s), b = __ldg(s + 1), c = __ldg(s + 2), d = __ldg(s + 3), e = __ldg(s + 4);
  q.p = df64(a.x, a.y); q.o2p = df64(a.z, a.w);
  q.P[0] = df64(b.x, b.y); q.P[1] = df64(b.z, b.w); q.P[2] = df64(c.x, c.y);
  q.PA[0] = df64(c.z, c.w); q.PA[1] = df64(d.x, d.y); q.PA[2] = df64(d.z, d.w);
  q.K = df64(e.x, e.y);
}

template <class C>
__device__ __forceinline__ void contracted_vrr_df(const PairSet& ps, const KernelCommon& kc, int b0, int nb, int k0,
                                                  int nk, df64* acc) {
#pragma unroll
  for (int x = 0; x < C::NE * C::NF; ++x) acc[x] = df64(0.0f, 0.0f);
  for (int ik = 0; ik < nk; ++ik) {
    Prim<df64> c;
    load_prim_df(ps.primdf, k0 + ik, c);
    for (int ib = 0; ib < nb; ++ib) {
      Prim<df64> a;
      load_prim_df(ps.primdf, b0 + ib, a);
      const df64 pq = a.p + c.p;
      const df64 rs = rsqrt(pq);
      const df64 inv = rs * rs;
      const df64 rp = c.p * inv;  // rho / zeta
      const df64 rq = a.p * inv;  // rho / eta
      df64 PQ[3], WP[3], WQ[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        PQ[i] = a.P[i] - c.P[i];
        WP[i] = -(rp * PQ[i]);
        WQ[i] = rq * PQ[i];
      }
      const df64 T = a.p * rp * (PQ[0] * PQ[0] + PQ[1] * PQ[1] + PQ[2] * PQ[2]);
      df64 B[C::L + 1];
      boys_df<C::L>(T, kc.boysdf, B);
      const df64 pref = a.K * c.K * rs;
#pragma unroll
      for (int m = 0; m <= C::L; ++m) B[m] = B[m] * pref;
      C::template vrr<df64>(acc, B, a.PA, WP, c.PA, WQ, a.o2p, c.o2p, df_scale2(inv, 0.5f), rp, rq);
    }
  }
}

// Cartesian component scale relative to the axial component,
// sqrt((2l-1)!! / ((2x-1)!! (2y-1)!! (2z-1)!!)), components ordered x power
// descending then y: d xy, xz, yz carry sqrt(3); f xyz sqrt(15), the
// mixed ones sqrt(5); g x^2yz-type sqrt(35), x^2y^2-type sqrt(35/3),
// x^3y-type sqrt(7); s, p and the axial components 1.
__device__ __forceinline__ constexpr double comp_scale(int l, int c) {
  return l == 2   ? ((c == 1 || c == 2 || c == 4) ? 1.7320508075688772935 : 1.0)
         : l == 3 ? (c == 4 ? 3.8729833462074168852 : (c == 0 || c == 6 || c == 9) ? 1.0 : 2.2360679774997896964)
         : l == 4 ? ((c == 0 || c == 10 || c == 14)  ? 1.0
                     : (c == 4 || c == 7 || c == 8)  ? 5.9160797830996160426
                     : (c == 3 || c == 5 || c == 12) ? 3.4156502553198660478
                                                     : 2.6457513110645905905)
                  : 1.0;
}

// Classes evaluated by Rys quadrature in the thread-per-quartet kernel
// declare RYS = true (rys.cu); the generated classes do not.
template <class C, class = void>
struct IsRys : std::false_type {};
template <class C>
struct IsRys<C, std::void_t<decltype(C::RYS)>> : std::integral_constant<bool, C::RYS> {};

__host__ __device__ constexpr int cart_power(int l, int c, int dir) {
  int k = 0;
  for (int x = l; x >= 0; --x)
    for (int y = l - x; y >= 0; --y) {
      if (k == c) return dir == 0 ? x : (dir == 1 ? y : l - x - y);
      ++k;
    }
  return 0;
}
__host__ __device__ constexpr double binom_c(int n, int k) {
  double r = 1.0;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return r;
}

// Contracted block of a small class by Rys quadrature, one quartet per lane
// (the recurrences of rys.cu with every size known at compile time, so the
// tables stay in registers): over the bra primitive pairs [ib0, ib1) and
// all ket primitives, per root the three G(n, m) tables, the transfer to
// B and D, and the Ix Iy Iz products, into I[(a NB + b) NC ND + c ND + d]
// (component scales not applied).  Inactive lanes return zeros.
template <class C>
__device__ __forceinline__ void rys_thread_block(const PairSet& P, const KernelCommon& kc, const PairInfo& bra,
                                                 const PairInfo& ket, int ib0, int ib1, bool active, double* I) {
  constexpr int LA = C::LA, LB = C::LB, LC = C::LC, LD = C::LD;
  constexpr int NA = C::NA, NB = C::NB, NC = C::NC, ND = C::ND;
  constexpr int NMAX = LA + LB, MMAX = LC + LD, NR = (LA + LB + LC + LD) / 2 + 1;
  constexpr int S4 = (LA + 1) * (LB + 1) * (LC + 1) * (LD + 1);
#pragma unroll
  for (int o = 0; o < NA * NB * NC * ND; ++o) I[o] = 0.0;
  if (!active) return;
  double ABp[3][LB + 1], CDp[3][LD + 1];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    ABp[d][0] = 1.0;
    CDp[d][0] = 1.0;
#pragma unroll
    for (int k = 1; k <= LB; ++k) ABp[d][k] = ABp[d][k - 1] * bra.AB[d];
#pragma unroll
    for (int k = 1; k <= LD; ++k) CDp[d][k] = CDp[d][k - 1] * ket.AB[d];
  }
  const int nk = ket.nprim;
  for (int ib = ib0; ib < ib1; ++ib) {
    const double* rb = P.prim64 + (size_t)(bra.prim0 + ib) * PRIM64_STRIDE;
    const double p = __ldg(rb), hp = __ldg(rb + 1);
    const double Pp[3] = {__ldg(rb + 2), __ldg(rb + 3), __ldg(rb + 4)};
    const double PA[3] = {__ldg(rb + 5), __ldg(rb + 6), __ldg(rb + 7)};
    const double Kab = __ldg(rb + 8);
    for (int ik = 0; ik < nk; ++ik) {
      const double* rk = P.prim64 + (size_t)(ket.prim0 + ik) * PRIM64_STRIDE;
      const double q = __ldg(rk), hq = __ldg(rk + 1);
      const double PQ[3] = {Pp[0] - __ldg(rk + 2), Pp[1] - __ldg(rk + 3), Pp[2] - __ldg(rk + 4)};
      const double QC[3] = {__ldg(rk + 5), __ldg(rk + 6), __ldg(rk + 7)};
      const double ipq = 1.0 / (p + q);
      const double T = p * q * ipq * (PQ[0] * PQ[0] + PQ[1] * PQ[1] + PQ[2] * PQ[2]);
      const double pref = Kab * __ldg(rk + 8) * sqrt(ipq);
      const double qf = q * ipq, pf = p * ipq;
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        double u, w;
        rys_rule_root(kc.rys, NR, r, T, &u, &w);
        const double B00 = 0.5 * u * ipq, B10 = hp * (1.0 - u * qf), B01 = hq * (1.0 - u * pf);
        double X[3][S4];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          double G[NMAX + 1][MMAX + 1];
          const double c00 = PA[d] - u * qf * PQ[d], d00 = QC[d] + u * pf * PQ[d];
          G[0][0] = d == 2 ? w * pref : 1.0;
#pragma unroll
          for (int n = 0; n < NMAX; ++n) G[n + 1][0] = c00 * G[n][0] + (n > 0 ? n * B10 * G[n - 1][0] : 0.0);
#pragma unroll
          for (int m = 0; m < MMAX; ++m)
#pragma unroll
            for (int n = 0; n <= NMAX; ++n)
              G[n][m + 1] = d00 * G[n][m] + (m > 0 ? m * B01 * G[n][m - 1] : 0.0) + (n > 0 ? n * B00 * G[n - 1][m] : 0.0);
#pragma unroll
          for (int ia = 0; ia <= LA; ++ia)
#pragma unroll
            for (int jb = 0; jb <= LB; ++jb)
#pragma unroll
              for (int ic = 0; ic <= LC; ++ic)
#pragma unroll
                for (int jd = 0; jd <= LD; ++jd) {
                  double v = 0.0;
#pragma unroll
                  for (int k = 0; k <= jb; ++k)
#pragma unroll
                    for (int l = 0; l <= jd; ++l)
                      v += binom_c(jb, k) * binom_c(jd, l) * ABp[d][jb - k] * CDp[d][jd - l] * G[ia + k][ic + l];
                  X[d][((ia * (LB + 1) + jb) * (LC + 1) + ic) * (LD + 1) + jd] = v;
                }
        }
#pragma unroll
        for (int a = 0; a < NA; ++a)
#pragma unroll
          for (int b = 0; b < NB; ++b)
#pragma unroll
            for (int c = 0; c < NC; ++c)
#pragma unroll
              for (int dd = 0; dd < ND; ++dd) {
                const int o = ((a * NB + b) * NC + c) * ND + dd;
                const int ix = ((cart_power(LA, a, 0) * (LB + 1) + cart_power(LB, b, 0)) * (LC + 1) + cart_power(LC, c, 0)) * (LD + 1) + cart_power(LD, dd, 0);
                const int iy = ((cart_power(LA, a, 1) * (LB + 1) + cart_power(LB, b, 1)) * (LC + 1) + cart_power(LC, c, 1)) * (LD + 1) + cart_power(LD, dd, 1);
                const int iz = ((cart_power(LA, a, 2) * (LB + 1) + cart_power(LB, b, 2)) * (LC + 1) + cart_power(LC, c, 2)) * (LD + 1) + cart_power(LD, dd, 2);
                I[o] = fma(X[0][ix] * X[1][iy], X[2][iz], I[o]);
              }
      }
    }
  }
}

// One contribution v to element idx of an accumulator.  Default: an FP64
// atomic add into base[idx].  Deterministic mode (HF_JK_DETERMINISTIC): base
// holds two 64-bit integers per element and v goes in as fixed point,
// hi = trunc(v 2^20) and lo = rint((v 2^20 - hi) 2^36), with integer atomic
// adds; integer addition is associative, so the sums, and J and K after
// the conversion back (hi 2^-20 + lo 2^-56), do not depend on the order in
// which the warps finish.  Resolution 2^-57 per contribution; lo stays in
// range for up to 2^27 contributions to one element.
__device__ __forceinline__ void jk_acc(double* base, size_t idx, double v, int det) {
  if (!det) {
    atomicAdd(base + idx, v);
    return;
  }
  unsigned long long* q = reinterpret_cast<unsigned long long*>(base) + 2 * idx;
  const double sc = v * 1048576.0;  // 2^20
  const double h = trunc(sc);
  const long long hi = (long long)h;
  const long long lo = __double2ll_rn((sc - h) * 68719476736.0);  // 2^36
  if (hi) atomicAdd(q, (unsigned long long)hi);
  if (lo) atomicAdd(q + 1, (unsigned long long)lo);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ------------------------------------------------------------- J/K kernel
// items: work item t covers bra list entry bi (found by binary search in
// ioff) and kets kbeg[bi] + 32*(t - ioff[bi]) + lane of the ket list.
// one: D/J/K of a single molecule (pair data ps, ket list w.ket); mols (if
// not null): per-molecule table indexed by w.mol[entry], each molecule with
// its own pair data, ket lists and D/J/K.
template <class C, typename R>
__global__ void __launch_bounds__(128) eri_jk_kernel(const JKWork w, const PairSet ps, const KernelCommon kc,
                                                     const MolJK one, const MolJK* __restrict__ mols) {
  constexpr int NA = C::NA, NB = C::NB, NC = C::NC, ND = C::ND;
  const int lane = threadIdx.x & 31;
  for (;;) {
    int t = 0;
    if (lane == 0) t = atomicAdd(w.counter, 1);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= w.nitems) break;
    int lo = 0, hi = w.nbra;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (__ldg(w.ioff + mid) <= t) lo = mid; else hi = mid;
    }
    const int bi = lo;
    const MolJK* mjp = mols ? mols + __ldg(w.mol + bi) : nullptr;
    if (mjp && !mjp->active) continue;  // warp-uniform: the entry is shared by the warp
    const PairSet P = mjp ? mjp->ps : ps;
    const int* ketb = mjp ? mjp->ketlist + mjp->ket_off[pair_class(C::LC, C::LD)] : w.ket;
    const int bp = __ldg(w.bra + bi);
    const int nsp = w.nsplit ? __ldg(w.nsplit + bi) : 1;
    const int rr = t - __ldg(w.ioff + bi);
    const int kblk = rr / nsp, part = rr - kblk * nsp;
    const int kidx = __ldg(w.kbeg + bi) + 32 * kblk + lane;
    if (!HF_BCHECK(kc, bp >= 0 && bp < P.npairs, HF_BC_PAIR, bp)) continue;
    bool active = kidx < __ldg(w.kend + bi);
    if (active && !HF_BCHECK(kc, kidx >= 0, HF_BC_ITEM, kidx)) active = false;
    int kp = active ? __ldg(ketb + kidx) : bp;
    if (active && !HF_BCHECK(kc, kp >= 0 && kp < P.npairs, HF_BC_PAIR, kp)) {
      active = false;
      kp = bp;
    }
    const PairInfo bra = P.info[bp];
    const PairInfo ket = P.info[kp];
    {
      const int nbf_ = mjp ? mjp->nbf : one.nbf;
      (void)nbf_;
      const bool bra_ok = HF_BCHECK(kc, bra.prim0 >= 0 && bra.prim0 + bra.nprim <= P.nprimpairs, HF_BC_PRIM,
                                    bra.prim0) &&
                          HF_BCHECK(kc, bra.bfA + NA <= nbf_ && bra.bfB + NB <= nbf_, HF_BC_MAT, bra.bfA);
      if (!bra_ok) continue;  // warp-uniform
      if (active && !(HF_BCHECK(kc, ket.prim0 >= 0 && ket.prim0 + ket.nprim <= P.nprimpairs, HF_BC_PRIM,
                                ket.prim0) &&
                      HF_BCHECK(kc, ket.bfA + NC <= nbf_ && ket.bfB + ND <= nbf_, HF_BC_MAT, ket.bfA)))
        active = false;
    }
    // this part's bra primitive pairs (all of them unless the item is split;
    // the contraction is linear, so the parts' digested blocks add up)
    const int ib0 = part * bra.nprim / nsp, ib1 = (part + 1) * bra.nprim / nsp;

    R I[NA * NB * NC * ND];
    if constexpr (IsRys<C>::value) {
      static_assert(std::is_same<R, double>::value, "Rys thread classes run in FP64");
      rys_thread_block<C>(P, kc, bra, ket, ib0, ib1, active, I);
    } else {
      R acc[C::NE * C::NF];
      if constexpr (std::is_same<R, df64>::value)
        contracted_vrr_df<C>(P, kc, bra.prim0 + ib0, ib1 - ib0, ket.prim0, active ? ket.nprim : 0, acc);
      else
        contracted_vrr<C, R>(P, kc, bra.prim0 + ib0, ib1 - ib0, ket.prim0, active ? ket.nprim : 0, acc);
      R AB[3] = {(R)bra.AB[0], (R)bra.AB[1], (R)bra.AB[2]};
      R CD[3] = {(R)ket.AB[0], (R)ket.AB[1], (R)ket.AB[2]};
      C::template hrr<R>(acc, I, AB, CD);
    }
    const MolJK& mo = mjp ? *mjp : one;
    const double* __restrict__ Dj = mo.Dj ? mo.Dj : mo.D;
    double* __restrict__ J = mo.J;
    const int nbf = mo.nbf;
    const int nspin = mo.D2 ? 2 : 1;
    // digestion arithmetic: FP32 for the reduced-precision quartets (their
    // integrals carry FP32 error already), FP64 otherwise; every sum is added
    // into the FP64 J and K
    using A = typename std::conditional<std::is_same<R, float>::value, float, double>::type;
    A wdeg = active ? (A)1 : (A)0;
    if (bra.same) wdeg *= (A)0.5;
    if (ket.same) wdeg *= (A)0.5;
    if (bp == kp) wdeg *= (A)0.5;

    const int a0 = bra.bfA, b0 = bra.bfB, c0 = ket.bfA, d0 = ket.bfB;
    // J'_ab = w sum_cd I D_cd  (warp-reduced: the bra is uniform over the warp)
    A Dcd[NC * ND];
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
      for (int d = 0; d < ND; ++d)
        Dcd[c * ND + d] = active ? (A)__ldg(Dj + (size_t)(c0 + c) * nbf + d0 + d) * (A)comp_scale(C::LC, c) * (A)comp_scale(C::LD, d) : (A)0;
#pragma unroll
    for (int a = 0; a < NA; ++a)
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        A s = (A)0;
#pragma unroll
        for (int cd = 0; cd < NC * ND; ++cd) s = fma((A)I[(a * NB + b) * NC * ND + cd], Dcd[cd], s);
        s = warp_sum(s * wdeg);
        if (lane == 0 && s != 0.0)
          jk_acc(J, (size_t)(a0 + a) * nbf + b0 + b, (double)(s * (A)comp_scale(C::LA, a) * (A)comp_scale(C::LB, b)), kc.det);
      }
    if (!active) continue;
    // J'_cd = w sum_ab I D_ab
    A Dab[NA * NB];
#pragma unroll
    for (int a = 0; a < NA; ++a)
#pragma unroll
      for (int b = 0; b < NB; ++b)
        Dab[a * NB + b] = (A)__ldg(Dj + (size_t)(a0 + a) * nbf + b0 + b) * (A)comp_scale(C::LA, a) * (A)comp_scale(C::LB, b);
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
      for (int d = 0; d < ND; ++d) {
        A s = (A)0;
#pragma unroll
        for (int ab = 0; ab < NA * NB; ++ab) s = fma((A)I[ab * NC * ND + c * ND + d], Dab[ab], s);
        jk_acc(J, (size_t)(c0 + c) * nbf + d0 + d, (double)(s * wdeg * (A)comp_scale(C::LC, c) * (A)comp_scale(C::LD, d)), kc.det);
      }
    // exchange of each spin: K from D, and K2 from D2 in two-spin builds
#pragma unroll 1
    for (int sp = 0; sp < nspin; ++sp) {
    const double* __restrict__ D = sp ? mo.D2 : mo.D;
    double* __restrict__ Kx = sp ? mo.K2 : mo.K;
    // K'_ac = w sum_bd I D_bd ;  K'_ad = w sum_bc I D_bc
    {
      A Dbd[NB * ND], Dbc[NB * NC];
#pragma unroll
      for (int b = 0; b < NB; ++b) {
#pragma unroll
        for (int d = 0; d < ND; ++d)
          Dbd[b * ND + d] = (A)__ldg(D + (size_t)(b0 + b) * nbf + d0 + d) * (A)comp_scale(C::LB, b) * (A)comp_scale(C::LD, d);
#pragma unroll
        for (int c = 0; c < NC; ++c)
          Dbc[b * NC + c] = (A)__ldg(D + (size_t)(b0 + b) * nbf + c0 + c) * (A)comp_scale(C::LB, b) * (A)comp_scale(C::LC, c);
      }
#pragma unroll
      for (int a = 0; a < NA; ++a) {
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          A s = (A)0;
#pragma unroll
          for (int b = 0; b < NB; ++b)
#pragma unroll
            for (int d = 0; d < ND; ++d) s = fma((A)I[((a * NB + b) * NC + c) * ND + d], Dbd[b * ND + d], s);
          jk_acc(Kx, (size_t)(a0 + a) * nbf + c0 + c, (double)(s * wdeg * (A)comp_scale(C::LA, a) * (A)comp_scale(C::LC, c)), kc.det);
        }
#pragma unroll
        for (int d = 0; d < ND; ++d) {
          A s = (A)0;
#pragma unroll
          for (int b = 0; b < NB; ++b)
#pragma unroll
            for (int c = 0; c < NC; ++c) s = fma((A)I[((a * NB + b) * NC + c) * ND + d], Dbc[b * NC + c], s);
          jk_acc(Kx, (size_t)(a0 + a) * nbf + d0 + d, (double)(s * wdeg * (A)comp_scale(C::LA, a) * (A)comp_scale(C::LD, d)), kc.det);
        }
      }
    }
    // K'_bc = w sum_ad I D_ad ;  K'_bd = w sum_ac I D_ac
    {
      A Dad[NA * ND], Dac[NA * NC];
#pragma unroll
      for (int a = 0; a < NA; ++a) {
#pragma unroll
        for (int d = 0; d < ND; ++d)
          Dad[a * ND + d] = (A)__ldg(D + (size_t)(a0 + a) * nbf + d0 + d) * (A)comp_scale(C::LA, a) * (A)comp_scale(C::LD, d);
#pragma unroll
        for (int c = 0; c < NC; ++c)
          Dac[a * NC + c] = (A)__ldg(D + (size_t)(a0 + a) * nbf + c0 + c) * (A)comp_scale(C::LA, a) * (A)comp_scale(C::LC, c);
      }
#pragma unroll
      for (int b = 0; b < NB; ++b) {
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          A s = (A)0;
#pragma unroll
          for (int a = 0; a < NA; ++a)
#pragma unroll
            for (int d = 0; d < ND; ++d) s = fma((A)I[((a * NB + b) * NC + c) * ND + d], Dad[a * ND + d], s);
          jk_acc(Kx, (size_t)(b0 + b) * nbf + c0 + c, (double)(s * wdeg * (A)comp_scale(C::LB, b) * (A)comp_scale(C::LC, c)), kc.det);
        }
#pragma unroll
        for (int d = 0; d < ND; ++d) {
          A s = (A)0;
#pragma unroll
          for (int a = 0; a < NA; ++a)
#pragma unroll
            for (int c = 0; c < NC; ++c) s = fma((A)I[((a * NB + b) * NC + c) * ND + d], Dac[a * NC + c], s);
          jk_acc(Kx, (size_t)(b0 + b) * nbf + d0 + d, (double)(s * wdeg * (A)comp_scale(C::LB, b) * (A)comp_scale(C::LD, d)), kc.det);
        }
      }
    }
    }  // spin
  }
}

// ------------------------------------------------------------- cooperative kernel
// df64 hooks of the generic (cooperative) kernel
__device__ __forceinline__ void load_prim(const float* __restrict__ base, int idx, Prim<df64>& q) {
  load_prim_df(base, idx, q);
}
template <> struct PrimBase<df64> { static __device__ __forceinline__ const float* get(const PairSet& s) { return s.primdf; } };
template <int L>
struct BoysSel<L, df64> {
  static __device__ __forceinline__ void eval(df64 T, const KernelCommon& kc, df64* F) { boys_df<L>(T, kc.boysdf, F); }
};

// a * b + c, fused in each arithmetic type of the cooperative kernel (the
// df64 one sits beside df_fma, where argument-dependent lookup finds it)
__device__ __forceinline__ double fmac(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fmac(float a, float b, float c) { return fmaf(a, b, c); }

// Classes with L >= 5: one warp per contracted quartet.  The primitive
// quartets are set up G at a time, one per lane: each lane forms its
// coefficient vector (PA, WP, QC, WQ, rho/p, rho/q, k/(2p), k/(2q),
// k/(2(p+q))) and B_m = prefactor * F_m in a row of shared memory.  The
// warp then takes the rows in order: B_m goes to the first VRR slots, the
// lanes evaluate the generated VRR node list level by level (node =
// c0 x0 + c1 x1 [+ c2 (x2 - c3 x3)] [+ c4 x4] over slots, c from the row,
// the bracketed terms as the node's type bits say), and
// lane l adds the targets l, l+32, ... into its registers.  After the
// primitive loop the contracted [e0|f0] go to shared memory, the bra HRR
// runs one f per lane, the ket HRR one ab per lane, and each of the six
// digestion contractions gives one output element per lane.
template <class C>
struct CoopSizes {
  static constexpr int NT = C::NE * C::NF;
  static constexpr int NAB = C::NA * C::NB, NCD = C::NC * C::ND;
  static constexpr int ROW = HF_NCOEF + C::L + 1;  // one primitive quartet's coefficients and B_m
  static constexpr int WS_HRR = NT + NAB * C::NF + NAB * NCD;
  __host__ __device__ static constexpr int ws(int g) { return C::NSLOT + g * ROW > WS_HRR ? C::NSLOT + g * ROW : WS_HRR; }  // words per warp
  // rows set up per pass: one per lane.  Measured on GB300 (60-atom s+p+d
  // molecule) 32 beats 16 and 8 in every class, (dd|dd) included although
  // its 124 KB per block then allow one block per SM: the serial part of
  // a primitive quartet, not occupancy, bounds these kernels.
  static constexpr int G_DEFAULT = 32;
};

__device__ __forceinline__ double comp_scale_rt(int l, int c) {
  return (l == 2 && (c == 1 || c == 2 || c == 4)) ? 1.7320508075688772935 : 1.0;
}

// The contracted Cartesian block of one shell quartet (bra|ket) over its
// primitive quartets [q_lo, q_hi), by one warp, in the scheme described
// above; on return the warp's shared memory s holds it after the [e0|f0]
// and the bra HRR rows: as doubles pre-multiplied by the d-component scales
// (R = double or df64) or as floats (R = float), at s + NT + NAB * NF.
template <class C, typename R, typename PB>
__device__ __forceinline__ void coop_block(const PB* __restrict__ pbase, const KernelCommon& kc, const PairInfo& bra,
                                           const PairInfo& ket, int q_lo, int nq, R* const s, const int G,
                                           const int lane) {
  using S = CoopSizes<C>;
  constexpr int NB = C::NB, NC = C::NC, ND = C::ND, NE = C::NE, NF = C::NF;
  constexpr int NT = S::NT, NAB = S::NAB, NCD = S::NCD, NK = (NT + 31) / 32;
  (void)NC;
  (void)ND;
  R* const stage = s + C::NSLOT;
  const uint4* __restrict__ nodes = hfgen::CoopTables<C>::nodes();
  const int* __restrict__ levels = hfgen::CoopTables<C>::levels();
  const unsigned short* __restrict__ tgt = hfgen::CoopTables<C>::targets();
  R acc[NK];
#pragma unroll
  for (int k = 0; k < NK; ++k) acc[k] = (R)0;
  for (int g0 = q_lo; g0 < nq; g0 += G) {
    const int q = g0 + lane;
    if (lane < G && q < nq) {
      const int ib = q / ket.nprim, ik = q - ib * ket.nprim;
      R* const cv = stage + lane * S::ROW;
      Prim<R> a, c;
      load_prim(pbase, bra.prim0 + ib, a);
      load_prim(pbase, ket.prim0 + ik, c);
      const R pq = a.p + c.p;
      const R rs = (R)rsqrt(pq);
      const R inv = rs * rs;
      const R rp = c.p * inv, rq = a.p * inv;
      R PQ[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        PQ[i] = a.P[i] - c.P[i];
        cv[1 + i] = a.PA[i];
        cv[4 + i] = -rp * PQ[i];
        cv[7 + i] = c.PA[i];
        cv[10 + i] = rq * PQ[i];
      }
      cv[0] = (R)0;
      cv[13] = rp;
      cv[14] = rq;
      const R o2pq = (R)0.5 * inv;
#pragma unroll
      for (int k = 1; k <= 8; ++k) {
        cv[14 + k] = (R)k * a.o2p;
        cv[22 + k] = (R)k * c.o2p;
        cv[30 + k] = (R)k * o2pq;
      }
      const R T = a.p * rp * (PQ[0] * PQ[0] + PQ[1] * PQ[1] + PQ[2] * PQ[2]);
      R B[C::L + 1];
      BoysSel<C::L, R>::eval(T, kc, B);
      const R pref = a.K * c.K * rs;
#pragma unroll
      for (int m = 0; m <= C::L; ++m) cv[HF_NCOEF + m] = B[m] * pref;
    }
    __syncwarp();
    const int ng = min(G, nq - g0);  // rows set up in this pass
    for (int jq = 0; jq < ng; ++jq) {
      const R* const cv = stage + jq * S::ROW;
      if (lane <= C::L) s[lane] = cv[HF_NCOEF + lane];
      __syncwarp();
      for (int lev = 0; lev < C::NLEV; ++lev) {
        const int n1 = __ldg(levels + lev);
        for (int n = (lev == 0 ? 0 : __ldg(levels + lev - 1)) + lane; n < n1; n += 32) {
          const uint4 d = __ldg(nodes + n);
          const unsigned c = d.w;
          R v = fmac(cv[(c >> 6) & 63u], s[d.y & 0xffffu], cv[c & 63u] * s[d.x >> 16]);
          if (c & (1u << 30))
            v = fmac(cv[(c >> 12) & 63u], fmac(-cv[(c >> 18) & 63u], s[d.z & 0xffffu], s[d.y >> 16]), v);
          if (c & (1u << 31)) v = fmac(cv[(c >> 24) & 63u], s[d.z >> 16], v);
          s[d.x & 0xffffu] = v;
        }
        __syncwarp();
      }
#pragma unroll
      for (int k = 0; k < NK; ++k) {
        const int tt = lane + 32 * k;
        if (tt < NT) acc[k] += s[__ldg(tgt + tt)];
      }
      __syncwarp();
    }
  }
  // contracted [e0|f0] -> shared memory, then HRR
  R* const A = s;
  R* const H = s + NT;
  R* const I = H + NAB * NF;
  constexpr bool kPre = sizeof(R) == sizeof(double);      // R = double or df64
  double* const Id = reinterpret_cast<double*>(I);        // same storage when kPre
#pragma unroll
  for (int k = 0; k < NK; ++k) {
    const int tt = lane + 32 * k;
    if (tt < NT) A[tt] = acc[k];
  }
  __syncwarp();
  {
    const R AB[3] = {(R)bra.AB[0], (R)bra.AB[1], (R)bra.AB[2]};
    for (int f = lane; f < NF; f += 32) {
      R x[NE], y[NAB];
#pragma unroll
      for (int e = 0; e < NE; ++e) x[e] = A[e * NF + f];
      C::template hrr_bra_row<R>(x, y, AB);
#pragma unroll
      for (int ab = 0; ab < NAB; ++ab) H[ab * NF + f] = y[ab];
    }
  }
  __syncwarp();
  {
    const R CD[3] = {(R)ket.AB[0], (R)ket.AB[1], (R)ket.AB[2]};
    for (int ab = lane; ab < NAB; ab += 32) {
      R x[NF], y[NCD];
#pragma unroll
      for (int f = 0; f < NF; ++f) x[f] = H[ab * NF + f];
      C::template hrr_ket_row<R>(x, y, CD);
      if constexpr (kPre) {
        // FP64 and df64: stored once as a double, already multiplied by the
        // d-component scales s_a s_b s_c s_d that every contraction needs
        const double sab = comp_scale_rt(C::LA, ab / NB) * comp_scale_rt(C::LB, ab % NB);
#pragma unroll
        for (int cd = 0; cd < NCD; ++cd)
          Id[ab * NCD + cd] = (double)y[cd] * (sab * comp_scale_rt(C::LC, cd / ND) * comp_scale_rt(C::LD, cd % ND));
      } else {
#pragma unroll
        for (int cd = 0; cd < NCD; ++cd) I[ab * NCD + cd] = y[cd];
      }
    }
  }
}

template <class C, typename R>
__global__ void __launch_bounds__(128) eri_jk_coop_kernel(const JKWork w, const PairSet ps, const KernelCommon kc,
                                                          const MolJK one, const MolJK* __restrict__ mols,
                                                          const int G) {
  using S = CoopSizes<C>;
  constexpr int NB = C::NB, NC = C::NC, ND = C::ND, NE = C::NE, NF = C::NF;
  constexpr int NT = S::NT, NAB = S::NAB, NCD = S::NCD;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* const s = reinterpret_cast<R*>(smem_raw) + (threadIdx.x >> 5) * S::ws(G);
  const int lane = threadIdx.x & 31;
  const auto* base = PrimBase<R>::get(ps);
  for (;;) {
    int t = 0;
    if (lane == 0) t = atomicAdd(w.counter, 1);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= w.nitems) break;
    int lo = 0, hi = w.nbra;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (__ldg(w.ioff + mid) <= t) lo = mid; else hi = mid;
    }
    const int bi = lo;
    const MolJK* mjp = mols ? mols + __ldg(w.mol + bi) : nullptr;
    if (mjp && !mjp->active) continue;
    const PairSet P = mjp ? mjp->ps : ps;
    const auto* pbase = mjp ? PrimBase<R>::get(mjp->ps) : base;
    const int* ketb = mjp ? mjp->ketlist + mjp->ket_off[pair_class(C::LC, C::LD)] : w.ket;
    const int bp = __ldg(w.bra + bi);
    const int nsp = w.nsplit ? __ldg(w.nsplit + bi) : 1;
    const int rr = t - __ldg(w.ioff + bi);
    const int kj = rr / nsp, part = rr - kj * nsp;
    const int kp = __ldg(ketb + __ldg(w.kbeg + bi) + kj);
    if (!HF_BCHECK(kc, bp >= 0 && bp < P.npairs, HF_BC_PAIR, bp)) continue;
    if (!HF_BCHECK(kc, kp >= 0 && kp < P.npairs, HF_BC_PAIR, kp)) continue;
    const PairInfo bra = P.info[bp];
    const PairInfo ket = P.info[kp];
    {
      const int nbf_ = mjp ? mjp->nbf : one.nbf;
      (void)nbf_;
      const bool ok =
          HF_BCHECK(kc, bra.prim0 >= 0 && bra.prim0 + bra.nprim <= P.nprimpairs, HF_BC_PRIM, bra.prim0) &&
          HF_BCHECK(kc, ket.prim0 >= 0 && ket.prim0 + ket.nprim <= P.nprimpairs, HF_BC_PRIM, ket.prim0) &&
          HF_BCHECK(kc, bra.bfA + C::NA <= nbf_ && bra.bfB + NB <= nbf_, HF_BC_MAT, bra.bfA) &&
          HF_BCHECK(kc, ket.bfA + NC <= nbf_ && ket.bfB + ND <= nbf_, HF_BC_MAT, ket.bfA);
      if (!ok) continue;  // warp-uniform: one quartet per warp
    }
    // this part's primitive quartets (all unless the item is split; the
    // parts' digested blocks add up)
    const int nq_all = bra.nprim * ket.nprim;
    const int q_lo = part * nq_all / nsp, nq = (part + 1) * nq_all / nsp;
    coop_block<C, R>(pbase, kc, bra, ket, q_lo, nq, s, G, lane);
    R* const I = s + NT + NAB * NF;
    constexpr bool kPre = sizeof(R) == sizeof(double);      // R = double or df64
    double* const Id = reinterpret_cast<double*>(I);        // same storage when kPre
    __syncwarp();
    // digestion: one output element per lane for each of the six contractions
    const MolJK& mo = mjp ? *mjp : one;
    const double* __restrict__ Dj = mo.Dj ? mo.Dj : mo.D;
    double* __restrict__ J = mo.J;
    const int nbf = mo.nbf;
    const int nspin = mo.D2 ? 2 : 1;
    double wdeg = 1.0;
    if (bra.same) wdeg *= 0.5;
    if (ket.same) wdeg *= 0.5;
    if (bp == kp) wdeg *= 0.5;
    const int a0 = bra.bfA, b0 = bra.bfB, c0 = ket.bfA, d0 = ket.bfB;
    // digestion arithmetic: FP32 for the reduced-precision quartets, FP64
    // otherwise; every sum is added into the FP64 J and K
    using Dg = typename std::conditional<std::is_same<R, float>::value, float, double>::type;
    auto Dsc_of = [&](const double* __restrict__ Dm, int r0, int lr, int i, int c0_, int lc, int j) -> Dg {
      const Dg dv = (Dg)__ldg(Dm + (size_t)(r0 + i) * nbf + c0_ + j);
      if constexpr (kPre) return dv;
      else return dv * (Dg)comp_scale_rt(lr, i) * (Dg)comp_scale_rt(lc, j);
    };
    auto Dsc = [&](int r0, int lr, int i, int c0_, int lc, int j) { return Dsc_of(Dj, r0, lr, i, c0_, lc, j); };
    auto Iv = [&](int a, int b, int c, int d) -> Dg {
      if constexpr (kPre) return Id[((a * NB + b) * NC + c) * ND + d];
      else return (Dg)I[((a * NB + b) * NC + c) * ND + d];
    };
    // scale of an output element: in the pre-scaled forms all four
    // component scales are already inside the integrals
    auto osc = [&](int l1, int i, int l2, int j) -> Dg {
      return kPre ? (Dg)1 : (Dg)comp_scale_rt(l1, i) * (Dg)comp_scale_rt(l2, j);
    };
    for (int o = lane; o < NAB; o += 32) {  // J'_ab = w sum_cd I D_cd
      const int a = o / NB, b = o % NB;
      Dg acc2 = (Dg)0;
      for (int c = 0; c < NC; ++c)
        for (int d = 0; d < ND; ++d) acc2 = fma(Iv(a, b, c, d), Dsc(c0, C::LC, c, d0, C::LD, d), acc2);
      jk_acc(J, (size_t)(a0 + a) * nbf + b0 + b, (double)(acc2 * (Dg)wdeg * osc(C::LA, a, C::LB, b)), kc.det);
    }
    for (int o = lane; o < NCD; o += 32) {  // J'_cd = w sum_ab I D_ab
      const int c = o / ND, d = o % ND;
      Dg acc2 = (Dg)0;
      for (int a = 0; a < C::NA; ++a)
        for (int b = 0; b < NB; ++b) acc2 = fma(Iv(a, b, c, d), Dsc(a0, C::LA, a, b0, C::LB, b), acc2);
      jk_acc(J, (size_t)(c0 + c) * nbf + d0 + d, (double)(acc2 * (Dg)wdeg * osc(C::LC, c, C::LD, d)), kc.det);
    }
#pragma unroll 1
    for (int sp = 0; sp < nspin; ++sp) {  // exchange of each spin: K from D, K2 from D2
    const double* __restrict__ Dk = sp ? mo.D2 : mo.D;
    double* __restrict__ Kx = sp ? mo.K2 : mo.K;
    auto Dsk = [&](int r0, int lr, int i, int c0_, int lc, int j) { return Dsc_of(Dk, r0, lr, i, c0_, lc, j); };
    for (int o = lane; o < C::NA * NC; o += 32) {  // K'_ac = w sum_bd I D_bd
      const int a = o / NC, c = o % NC;
      Dg acc2 = (Dg)0;
      for (int b = 0; b < NB; ++b)
        for (int d = 0; d < ND; ++d) acc2 = fma(Iv(a, b, c, d), Dsk(b0, C::LB, b, d0, C::LD, d), acc2);
      jk_acc(Kx, (size_t)(a0 + a) * nbf + c0 + c, (double)(acc2 * (Dg)wdeg * osc(C::LA, a, C::LC, c)), kc.det);
    }
    for (int o = lane; o < C::NA * ND; o += 32) {  // K'_ad = w sum_bc I D_bc
      const int a = o / ND, d = o % ND;
      Dg acc2 = (Dg)0;
      for (int b = 0; b < NB; ++b)
        for (int c = 0; c < NC; ++c) acc2 = fma(Iv(a, b, c, d), Dsk(b0, C::LB, b, c0, C::LC, c), acc2);
      jk_acc(Kx, (size_t)(a0 + a) * nbf + d0 + d, (double)(acc2 * (Dg)wdeg * osc(C::LA, a, C::LD, d)), kc.det);
    }
    for (int o = lane; o < NB * NC; o += 32) {  // K'_bc = w sum_ad I D_ad
      const int b = o / NC, c = o % NC;
      Dg acc2 = (Dg)0;
      for (int a = 0; a < C::NA; ++a)
        for (int d = 0; d < ND; ++d) acc2 = fma(Iv(a, b, c, d), Dsk(a0, C::LA, a, d0, C::LD, d), acc2);
      jk_acc(Kx, (size_t)(b0 + b) * nbf + c0 + c, (double)(acc2 * (Dg)wdeg * osc(C::LB, b, C::LC, c)), kc.det);
    }
    for (int o = lane; o < NB * ND; o += 32) {  // K'_bd = w sum_ac I D_ac
      const int b = o / ND, d = o % ND;
      Dg acc2 = (Dg)0;
      for (int a = 0; a < C::NA; ++a)
        for (int c = 0; c < NC; ++c) acc2 = fma(Iv(a, b, c, d), Dsk(a0, C::LA, a, c0, C::LC, c), acc2);
      jk_acc(Kx, (size_t)(b0 + b) * nbf + d0 + d, (double)(acc2 * (Dg)wdeg * osc(C::LB, b, C::LD, d)), kc.det);
    }
    }  // spin
    __syncwarp();
  }
}

// Q_ab of the pairs of a warp-cooperative diagonal class (X|X): one warp per
// pair evaluates (ab|ab) by coop_block and takes sqrt(max |(ab|ab)|) over
// the Cartesian components (the thread-per-pair kernel below would hold
// the whole [e0|f0] set of these classes in registers).
template <class C>
__global__ void __launch_bounds__(128) eri_schwarz_coop_kernel(const int* __restrict__ pairs, int npairs,
                                                               const PairSet ps, const KernelCommon kc,
                                                               double* __restrict__ Q, const int G) {
  using S = CoopSizes<C>;
  constexpr int NT = S::NT, NAB = S::NAB, NCD = S::NCD, NF = C::NF;
  static_assert(NAB == NCD, "diagonal class");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* const s = reinterpret_cast<double*>(smem_raw) + (threadIdx.x >> 5) * S::ws(G);
  const int lane = threadIdx.x & 31;
  const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;  // one pair per warp
  if (t >= npairs) return;
  const int pid = pairs[t];
  const PairInfo pr = ps.info[pid];
  coop_block<C, double>(ps.prim64, kc, pr, pr, 0, pr.nprim * pr.nprim, s, G, lane);
  __syncwarp();
  const double* const Id = s + NT + NAB * NF;  // pre-scaled: (ab|ab) s_a^2 s_b^2
  double m = 0.0;
  for (int ab = lane; ab < NAB; ab += 32) m = fmax(m, fabs(Id[ab * NCD + ab]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) Q[pid] = sqrt(m);
}

// Primitive quartets set up per pass: the class default, or HF_COOP_G
// (8, 16 or 32) from the environment for tuning.
template <class C>
inline int coop_group() {
  static const int g = [] {
    const char* e = getenv("HF_COOP_G");
    const int v = e ? atoi(e) : 0;
    return (v == 8 || v == 16 || v == 32) ? v : CoopSizes<C>::G_DEFAULT;
  }();
  return g;
}

template <class C, typename R>
inline size_t coop_smem_bytes(int g) {
  return (size_t)4 * CoopSizes<C>::ws(g) * sizeof(R);
}

template <class C, typename R>
inline void coop_launch(const JKWork& w, const PairSet& ps, const KernelCommon& kc, const MolJK& one,
                        const MolJK* mols, int grid, int threads, cudaStream_t s) {
  const int g = coop_group<C>();
  const size_t sm = coop_smem_bytes<C, R>(g);
  static bool attr = false;  // set once per process (same function on every device)
  if (!attr) {
    cudaFuncSetAttribute(eri_jk_coop_kernel<C, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    attr = true;
  }
  // shared memory per warp of the block (the attribute covers four warps)
  const size_t used = sm / 4 * (size_t)(threads / 32);
  eri_jk_coop_kernel<C, R><<<grid, threads, used, s>>>(w, ps, kc, one, mols, g);
}

template <class C>
inline void schwarz_coop_launch(const int* pairs, int npairs, const PairSet& ps, const KernelCommon& kc, double* Q,
                                cudaStream_t s) {
  const int g = coop_group<C>();
  const size_t sm = coop_smem_bytes<C, double>(g);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(eri_schwarz_coop_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    attr = true;
  }
  eri_schwarz_coop_kernel<C><<<(npairs + 3) / 4, 128, sm, s>>>(pairs, npairs, ps, kc, Q, g);
}

template <class C, typename R>
inline int coop_occupancy() {
  const size_t sm = coop_smem_bytes<C, R>(coop_group<C>());
  cudaFuncSetAttribute(eri_jk_coop_kernel<C, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  int n = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, eri_jk_coop_kernel<C, R>, 128, sm);
  return n;
}

// ------------------------------------------------------------- ERI tensor kernel
// Same work decomposition; every element of the block is written to all
// eight index permutations of the dense nbf^4 tensor G (small bases).
template <class C>
__global__ void __launch_bounds__(128) eri_store_kernel(const JKWork w, const PairSet ps, const KernelCommon kc,
                                                        double* __restrict__ G, int nbf) {
  constexpr int NA = C::NA, NB = C::NB, NC = C::NC, ND = C::ND;
  const int lane = threadIdx.x & 31;
  for (;;) {
    int t = 0;
    if (lane == 0) t = atomicAdd(w.counter, 1);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= w.nitems) break;
    int lo = 0, hi = w.nbra;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (__ldg(w.ioff + mid) <= t) lo = mid; else hi = mid;
    }
    const int bi = lo;
    const int bp = __ldg(w.bra + bi);
    // the tensor is written, not accumulated: part 0 of a split item takes
    // the whole primitive loop and the other parts do nothing
    const int nsp = w.nsplit ? __ldg(w.nsplit + bi) : 1;
    const int rr = t - __ldg(w.ioff + bi);
    if (rr % nsp != 0) continue;
    const int kidx = __ldg(w.kbeg + bi) + w.chunk * (rr / nsp) + lane;
    if (lane >= w.chunk || kidx >= __ldg(w.kend + bi)) continue;
    const int kp = __ldg(w.ket + kidx);
    const PairInfo bra = ps.info[bp];
    const PairInfo ket = ps.info[kp];
    double acc[C::NE * C::NF];
    contracted_vrr<C, double>(ps, kc, bra.prim0, bra.nprim, ket.prim0, ket.nprim, acc);
    double I[NA * NB * NC * ND];
    C::template hrr<double>(acc, I, bra.AB, ket.AB);
    const size_t n = (size_t)nbf;
#pragma unroll
    for (int a = 0; a < NA; ++a)
#pragma unroll
      for (int b = 0; b < NB; ++b)
#pragma unroll
        for (int c = 0; c < NC; ++c)
#pragma unroll
          for (int d = 0; d < ND; ++d) {
            const double v = I[((a * NB + b) * NC + c) * ND + d] * comp_scale(C::LA, a) * comp_scale(C::LB, b) *
                             comp_scale(C::LC, c) * comp_scale(C::LD, d);
            const size_t i = bra.bfA + a, j = bra.bfB + b, k = ket.bfA + c, l = ket.bfB + d;
            G[((i * n + j) * n + k) * n + l] = v;
            G[((j * n + i) * n + k) * n + l] = v;
            G[((i * n + j) * n + l) * n + k] = v;
            G[((j * n + i) * n + l) * n + k] = v;
            G[((k * n + l) * n + i) * n + j] = v;
            G[((l * n + k) * n + i) * n + j] = v;
            G[((k * n + l) * n + j) * n + i] = v;
            G[((l * n + k) * n + j) * n + i] = v;
          }
  }
}

// ------------------------------------------------------------- Schwarz kernel
// Q_ab = sqrt(max over components |(ab|ab)|) for the pairs of one class;
// one thread per pair (bra = ket), pairs[] lists the pair ids.
template <class C>
__global__ void __launch_bounds__(128) eri_schwarz_kernel(const int* __restrict__ pairs, int npairs, const PairSet ps,
                                                          const KernelCommon kc, double* __restrict__ Q) {
  constexpr int NA = C::NA, NB = C::NB;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= npairs) return;
  const int pid = pairs[t];
  const PairInfo pr = ps.info[pid];
  double acc[C::NE * C::NF];
  contracted_vrr<C, double>(ps, kc, pr.prim0, pr.nprim, pr.prim0, pr.nprim, acc);
  double I[NA * NB * NA * NB];
  C::template hrr<double>(acc, I, pr.AB, pr.AB);
  double m = 0.0;
#pragma unroll
  for (int a = 0; a < NA; ++a)
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const double s = comp_scale(C::LA, a) * comp_scale(C::LB, b);
      const double v = fabs(I[((a * NB + b) * NA + a) * NB + b]) * s * s;
      m = v > m ? v : m;
    }
  Q[pid] = sqrt(m);
}

}  // namespace hfk

// Instantiate the launchers of one class into the dispatch table entry.
#define HF_DEFINE_CLASS_LAUNCHERS(CLS)                                                                   \
  template <typename R>                                                                                  \
  static void launch_jkR_##CLS(const JKWork& w, const PairSet& ps, const KernelCommon& kc, const MolJK& one,  \
                               const MolJK* mols, int grid, int threads, cudaStream_t s) {               \
    if constexpr (hfgen::CLS::COOP)                                                                      \
      hfk::coop_launch<hfgen::CLS, R>(w, ps, kc, one, mols, grid, threads, s);                           \
    else                                                                                                 \
      hfk::eri_jk_kernel<hfgen::CLS, R><<<grid, threads, 0, s>>>(w, ps, kc, one, mols);                  \
  }                                                                                                      \
  template <typename R>                                                                                  \
  static int occR_##CLS() {                                                                              \
    int n = 0;                                                                                           \
    if constexpr (hfgen::CLS::COOP)                                                                      \
      n = hfk::coop_occupancy<hfgen::CLS, R>();                                                          \
    else                                                                                                 \
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, hfk::eri_jk_kernel<hfgen::CLS, R>, 128, 0);      \
    return n;                                                                                            \
  }                                                                                                      \
  static void launch_jk64_##CLS(const JKWork& w, const PairSet& ps, const KernelCommon& kc, const MolJK& one, \
                                const MolJK* mols, int grid, int threads, cudaStream_t s) {              \
    launch_jkR_##CLS<double>(w, ps, kc, one, mols, grid, threads, s);                                    \
  }                                                                                                      \
  static void launch_jk32_##CLS(const JKWork& w, const PairSet& ps, const KernelCommon& kc, const MolJK& one, \
                                const MolJK* mols, int grid, int threads, cudaStream_t s) {              \
    launch_jkR_##CLS<float>(w, ps, kc, one, mols, grid, threads, s);                                     \
  }                                                                                                      \
  static void launch_jkdf_##CLS(const JKWork& w, const PairSet& ps, const KernelCommon& kc, const MolJK& one, \
                                const MolJK* mols, int grid, int threads, cudaStream_t s) {              \
    if constexpr (hfgen::CLS::COOP)                                                                      \
      hfk::coop_launch<hfgen::CLS, df64>(w, ps, kc, one, mols, grid, threads, s);                        \
    else if constexpr (hfgen::CLS::L <= HF_DF_LMAX)                                                      \
      hfk::eri_jk_kernel<hfgen::CLS, df64><<<grid, threads, 0, s>>>(w, ps, kc, one, mols);               \
    else                                                                                                 \
      launch_jkR_##CLS<double>(w, ps, kc, one, mols, grid, threads, s);                                  \
  }                                                                                                      \
  static int occ_jkdf_##CLS() {                                                                          \
    int n = 0;                                                                                           \
    if constexpr (hfgen::CLS::COOP)                                                                      \
      n = hfk::coop_occupancy<hfgen::CLS, df64>();                                                       \
    else if constexpr (hfgen::CLS::L <= HF_DF_LMAX)                                                      \
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, hfk::eri_jk_kernel<hfgen::CLS, df64>, 128, 0);   \
    else                                                                                                 \
      n = occR_##CLS<double>();                                                                          \
    return n;                                                                                            \
  }                                                                                                      \
  static void launch_store_##CLS(const JKWork& w, const PairSet& ps, const KernelCommon& kc, double* G,   \
                                 int nbf, int grid, cudaStream_t s) {                                    \
    hfk::eri_store_kernel<hfgen::CLS><<<grid, 128, 0, s>>>(w, ps, kc, G, nbf);                           \
  }                                                                                                      \
  static void launch_schwarz_##CLS(const int* pairs, int npairs, const PairSet& ps, const KernelCommon& kc, \
                                   double* Q, cudaStream_t s) {                                          \
    if (npairs <= 0) return;                                                                             \
    if constexpr (hfgen::CLS::COOP && hfgen::CLS::LA == hfgen::CLS::LC && hfgen::CLS::LB == hfgen::CLS::LD)  \
      hfk::schwarz_coop_launch<hfgen::CLS>(pairs, npairs, ps, kc, Q, s);                                  \
    else                                                                                                 \
      hfk::eri_schwarz_kernel<hfgen::CLS><<<(npairs + 127) / 128, 128, 0, s>>>(pairs, npairs, ps, kc, Q); \
  }                                                                                                      \
  static int occ_jk64_##CLS() { return occR_##CLS<double>(); }                                          \
  static int occ_jk32_##CLS() { return occR_##CLS<float>(); }

#define HF_REGISTER_CLASS(table, CLS, la, lb, lc, ld, vf, hf_)                                           \
  do {                                                                                                   \
    EriClassOps& e = table[class_index(la, lb, lc, ld)];                                                 \
    e.jk64 = launch_jk64_##CLS;                                                                          \
    e.jk32 = launch_jk32_##CLS;                                                                          \
    e.jkdf = launch_jkdf_##CLS;                                                                          \
    e.occdf = occ_jkdf_##CLS;                                                                            \
    e.store = launch_store_##CLS;                                                                        \
    e.schwarz = launch_schwarz_##CLS;                                                                    \
    e.occ64 = occ_jk64_##CLS;                                                                            \
    e.occ32 = occ_jk32_##CLS;                                                                            \
    e.chunk = hfgen::CLS::COOP ? 1 : 32;                                                                 \
    e.vrr_flops = vf;                                                                                    \
    e.hrr_flops = hf_;                                                                                   \
    e.name = #CLS;                                                                                       \
  } while (0)
