// rys.cuh -- the Rys quadrature rule behind the electron repulsion
// integrals of Eq. 5 (the paper evaluates them by Rys quadrature): the
// layout of the table of roots and weights, and its evaluation, shared by
// the device kernels (rys.cu, eri.cuh, onee.cu, grad.cu) and the host.
//
// The n-point Rys rule for a primitive quartet with T = rho |PQ|^2 is the
// Gauss rule of the weight exp(-T t^2) on t in [0, 1] in the variable
// u = t^2:
//     int_0^1 f(t^2) exp(-T t^2) dt = sum_i w_i f(u_i),
// exact for polynomials f of degree <= 2n - 1, so sum_i w_i u_i^k = F_k(T)
// (the Boys function) for k < 2n.  An ERI of total angular momentum L is a
// polynomial of degree floor(L/2) in u under that integral, so
// n = floor(L/2) + 1 roots make it exact.
//
// Table: for n = 1..RYS_NMAX and T in [0, RYS_TMAX), intervals of width
// 1 / RYS_INV_H; per interval and root a Chebyshev series of RYS_NCHEB
// terms for u_i(T) and one for w_i(T) in x = 2 RYS_INV_H (T - T_j) - 1.  For
// T >= RYS_TMAX the half-range Gauss-Hermite limit is used:
// u_i = s_i^2 / T and w_i = W_i / sqrt(T), with s_i > 0 the positive nodes
// and W_i the weights of the 2n-point Gauss-Hermite rule (the integral to
// infinity differs from the one to t = 1 by less than 1e-16 relative there
// for the degrees used).  The host builds the table once per process.
#pragma once

#include <cmath>

#define RYS_NMAX 9       // (gg|gg) has L = 16: 9 roots
#define RYS_NCHEB 10
#define RYS_NINT 120
#define RYS_INV_H 2.0    // 1 / interval width
#define RYS_TMAX 60.0

// offset of the n-point block: n (n - 1) / 2 earlier roots per interval
__host__ __device__ constexpr int rys_tab_off(int n) { return RYS_NINT * 2 * RYS_NCHEB * ((n - 1) * n / 2); }
#define RYS_ASYM_OFF rys_tab_off(RYS_NMAX + 1)
#define RYS_TAB_DOUBLES (RYS_ASYM_OFF + RYS_NMAX * (RYS_NMAX + 1))

// Chebyshev series sum_k c_k T_k(x) by Clenshaw's recurrence.
__host__ __device__ inline double rys_cheb(const double* c, double x) {
  double b1 = 0.0, b2 = 0.0;
  const double x2 = 2.0 * x;
  for (int k = RYS_NCHEB - 1; k >= 1; --k) {
    const double t = fma(x2, b1, c[k] - b2);
    b2 = b1;
    b1 = t;
  }
  return fma(x, b1, c[0] - b2);
}

// Root i (0-based, ascending) and weight of the n-point rule at T >= 0.
__host__ __device__ inline void rys_rule_root(const double* tab, int n, int i, double T, double* u, double* w) {
  if (!(T < RYS_TMAX)) {
    const double* a = tab + RYS_ASYM_OFF + 2 * (n * (n - 1) / 2 + i);
    *u = a[0] / T;
    *w = a[1] / sqrt(T);
    return;
  }
  int j = (int)(T * RYS_INV_H);
  j = j < 0 ? 0 : (j > RYS_NINT - 1 ? RYS_NINT - 1 : j);
  const double x = 2.0 * RYS_INV_H * T - (2 * j + 1);
  const double* c = tab + rys_tab_off(n) + (size_t)(j * n + i) * 2 * RYS_NCHEB;
  *u = rys_cheb(c, x);
  *w = rys_cheb(c + RYS_NCHEB, x);
}

// Host: the table (RYS_TAB_DOUBLES values), built on first use and kept for
// the process.  Thread-safe.
const double* hf_rys_table_host();
