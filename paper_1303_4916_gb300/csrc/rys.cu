// rys.cu -- the Rys-quadrature route for the ERIs of Eq. 5 (the paper's
// own route): the host-built table of Rys roots and weights, and one
// warp per contracted shell quartet for every class with an f or g shell
// (la..ld <= 4), or for all classes when HF_JK_RYS is set.
//
// Per primitive quartet (exponents a, b | c, d; p = a + b, q = c + d,
// P, Q the Gaussian-product centres, PA = P - A, QC = Q - C) and per root
// u of the n-point Rys rule at T = pq/(p+q) |PQ|^2, the integral factorises
// into three one-dimensional tables G(n, m) (n: power on A, m: power on C)
// built by the Rys recurrences
//     G(0, 0)      = 1 (x, y);  w * K'_ab K'_cd / sqrt(p+q) (z)
//     G(n+1, 0)    = C00 G(n, 0) + n B10 G(n-1, 0)
//     G(n, m+1)    = D00 G(n, m) + m B01 G(n, m-1) + n B00 G(n-1, m)
// with  B00 = u / (2 (p+q)),  B10 = (1 - u q/(p+q)) / (2p),
//       B01 = (1 - u p/(p+q)) / (2q),
//       C00 = PA - u q/(p+q) (P - Q),  D00 = QC + u p/(p+q) (P - Q),
// then moved to B and D by the transfer (x-B)^b = sum_k C(b,k) (x-A)^k
// (A-B)^(b-k) (and likewise for D on the ket):
//     I(ia, ib; ic, id) = sum_k C(ib,k) AB^(ib-k) sum_l C(id,l) CD^(id-l)
//                         G(ia + k, ic + l),
// and (ab|cd) = sum over roots and primitive quartets of Ix Iy Iz.
//
// One warp per work item: a chunk of one contracted quartet's output block
// (whole (a, b) rows, all c, d, at most 1024 outputs) over a range of its
// primitive quartets.  The G tables and both transfers live in the warp's
// slice of shared memory; each lane keeps up to 32 of the chunk's outputs
// in registers; the finished chunk is digested into J and K as the
// cooperative kernels do (same symmetry weights and accumulators).  The
// smallest f/g classes run one quartet per lane instead (rys_thread.cu).
// The gradient's derivative kernel (rys_grad_kernel) shares the tables,
// one power higher on A, B and C.
#include <algorithm>
#include <array>
#include <cfloat>
#include <cmath>
#include <mutex>
#include <utility>
#include <vector>

#include "eri.cuh"
#include "hf_internal.h"
#include "rys.cuh"

// ------------------------------------------------------------- host table
namespace {

typedef long double ld;

// Gauss-Legendre nodes and weights on [-1, 1] (Newton on the Legendre
// three-term recurrence).
void gauss_legendre(int M, std::vector<ld>& x, std::vector<ld>& w) {
  x.resize(M);
  w.resize(M);
  const ld pi = 3.141592653589793238462643383279502884L;
  for (int i = 0; i < M; ++i) {
    ld z = cosl(pi * (i + 0.75L) / (M + 0.5L)), dp = 1.0L;
    for (int it = 0; it < 100; ++it) {
      ld p0 = 1.0L, p1 = z;
      for (int k = 2; k <= M; ++k) {
        const ld p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = M * (z * p1 - p0) / (z * z - 1.0L);
      const ld dz = p1 / dp;
      z -= dz;
      if (fabsl(dz) <= 1e-4L * LDBL_EPSILON) break;
    }
    x[i] = z;
    w[i] = 2.0L / ((1.0L - z * z) * dp * dp);
  }
}

// Recurrence coefficients a_k, b_k (k < nmax) of the monic polynomials
// orthogonal under the discrete measure sum_j W_j f(u_j): discretised
// Stieltjes procedure, pi_{k+1} = (u - a_k) pi_k - b_k pi_{k-1},
// b_0 = sum_j W_j.
void stieltjes(const std::vector<ld>& u, const std::vector<ld>& W, int nmax, ld* a, ld* b) {
  const size_t M = u.size();
  std::vector<ld> pm(M, 0.0L), p(M, 1.0L);
  ld prev = 1.0L;
  for (int k = 0; k < nmax; ++k) {
    ld nrm = 0.0L, mom = 0.0L;
    for (size_t j = 0; j < M; ++j) {
      const ld t = W[j] * p[j] * p[j];
      nrm += t;
      mom += t * u[j];
    }
    a[k] = mom / nrm;
    b[k] = k == 0 ? nrm : nrm / prev;
    prev = nrm;
    for (size_t j = 0; j < M; ++j) {
      const ld pn = (u[j] - a[k]) * p[j] - (k > 0 ? b[k] * pm[j] : 0.0L);
      pm[j] = p[j];
      p[j] = pn;
    }
  }
}

// Gauss rule of n points from the recurrence: nodes are the eigenvalues of
// the Jacobi matrix (diagonal a_k, off-diagonal sqrt(b_k)), found by Sturm
// bisection in [lo, hi] and polished by Newton on pi_n; weights by the
// Christoffel formula w = 1 / sum_k pi_k(x)^2 / (b_0 ... b_k).
void gauss_rule(int n, const ld* a, const ld* b, ld lo0, ld hi0, ld* x, ld* w) {
  auto below = [&](ld z) {  // eigenvalues < z
    int c = 0;
    ld q = a[0] - z;
    if (q < 0) ++c;
    for (int k = 1; k < n; ++k) {
      if (q == 0) q = LDBL_MIN;
      q = a[k] - z - b[k] / q;
      if (q < 0) ++c;
    }
    return c;
  };
  auto pn = [&](ld z, ld* dp) {
    ld p0 = 0.0L, p1 = 1.0L, d0 = 0.0L, d1 = 0.0L;
    for (int k = 0; k < n; ++k) {
      const ld p2 = (z - a[k]) * p1 - (k > 0 ? b[k] * p0 : 0.0L);
      const ld d2 = p1 + (z - a[k]) * d1 - (k > 0 ? b[k] * d0 : 0.0L);
      p0 = p1;
      p1 = p2;
      d0 = d1;
      d1 = d2;
    }
    *dp = d1;
    return p1;
  };
  for (int i = 0; i < n; ++i) {
    ld lo = lo0, hi = hi0;
    for (int it = 0; it < 200; ++it) {  // to ~1e-9 relative, then Newton
      const ld mid = 0.5L * (lo + hi);
      if (mid == lo || mid == hi || hi - lo <= 1e-9L * fabsl(mid)) break;
      if (below(mid) > i) hi = mid; else lo = mid;
    }
    ld z = 0.5L * (lo + hi);
    for (int it = 0; it < 8; ++it) {
      ld dp;
      const ld f = pn(z, &dp);
      if (dp == 0) break;
      const ld zn = z - f / dp;
      if (!(zn > lo && zn < hi)) break;
      const ld dz = zn - z;
      z = zn;
      if (fabsl(dz) <= 2 * LDBL_EPSILON * fabsl(z)) break;
    }
    x[i] = z;
    ld s = 0.0L, pm = 0.0L, p = 1.0L, h = b[0];
    s = 1.0L / h;
    for (int k = 0; k + 1 < n; ++k) {
      const ld p2 = (z - a[k]) * p - (k > 0 ? b[k] * pm : 0.0L);
      pm = p;
      p = p2;
      h *= b[k + 1];
      s += p * p / h;
    }
    w[i] = 1.0L / s;
  }
}

std::vector<double> build_rys_table() {
  std::vector<double> tab(RYS_TAB_DOUBLES, 0.0);
  std::vector<ld> gx, gw;
  gauss_legendre(160, gx, gw);
  const int M = (int)gx.size();
  std::vector<ld> u(M), W(M);
  const ld pi = 3.141592653589793238462643383279502884L;
  ld cosk[RYS_NCHEB][RYS_NCHEB];
  for (int m = 0; m < RYS_NCHEB; ++m)
    for (int k = 0; k < RYS_NCHEB; ++k) cosk[m][k] = cosl(pi * m * (k + 0.5L) / RYS_NCHEB);
  // rule values at the Chebyshev nodes of every interval, all n at once
  std::vector<ld> val((size_t)RYS_NINT * RYS_NCHEB * RYS_NMAX * 2 * RYS_NMAX);  // [j][k][n-1][2 RYS_NMAX]
  auto vidx = [&](int j, int k, int n) { return (((size_t)j * RYS_NCHEB + k) * RYS_NMAX + (n - 1)) * 2 * RYS_NMAX; };
  for (int j = 0; j < RYS_NINT; ++j)
    for (int k = 0; k < RYS_NCHEB; ++k) {
      const ld xk = cosl(pi * (k + 0.5L) / RYS_NCHEB);
      const ld T = (j + 0.5L * (xk + 1.0L)) / (ld)RYS_INV_H;
      for (int i = 0; i < M; ++i) {
        const ld t = 0.5L * (gx[i] + 1.0L);
        u[i] = t * t;
        W[i] = 0.5L * gw[i] * expl(-T * t * t);
      }
      ld a[RYS_NMAX], b[RYS_NMAX];
      stieltjes(u, W, RYS_NMAX, a, b);
      for (int n = 1; n <= RYS_NMAX; ++n) {
        ld x[RYS_NMAX], w[RYS_NMAX];
        gauss_rule(n, a, b, 0.0L, 1.0L, x, w);
        ld* v = val.data() + vidx(j, k, n);
        for (int i = 0; i < n; ++i) {
          v[2 * i] = x[i];
          v[2 * i + 1] = w[i];
        }
      }
    }
  for (int n = 1; n <= RYS_NMAX; ++n)
    for (int j = 0; j < RYS_NINT; ++j)
      for (int i = 0; i < n; ++i)
        for (int f = 0; f < 2; ++f) {
          double* c = tab.data() + rys_tab_off(n) + (size_t)(j * n + i) * 2 * RYS_NCHEB + f * RYS_NCHEB;
          for (int m = 0; m < RYS_NCHEB; ++m) {
            ld s = 0.0L;
            for (int k = 0; k < RYS_NCHEB; ++k) s += val[vidx(j, k, n) + 2 * i + f] * cosk[m][k];
            s *= 2.0L / RYS_NCHEB;
            if (m == 0) s *= 0.5L;
            c[m] = (double)s;
          }
        }
  // large-T limit: positive nodes s_i and weights of the 2n-point
  // Gauss-Hermite rule (monic recurrence a_k = 0, b_k = k / 2, b_0 = sqrt(pi))
  for (int n = 1; n <= RYS_NMAX; ++n) {
    const int m2 = 2 * n;
    ld a[2 * RYS_NMAX], b[2 * RYS_NMAX], x[2 * RYS_NMAX], w[2 * RYS_NMAX];
    for (int k = 0; k < m2; ++k) {
      a[k] = 0.0L;
      b[k] = k == 0 ? sqrtl(pi) : 0.5L * k;
    }
    const ld bound = 2.0L * sqrtl((ld)m2) + 2.0L;
    gauss_rule(m2, a, b, -bound, bound, x, w);
    for (int i = 0; i < n; ++i) {  // ascending: the upper half is the positive nodes
      const ld s = x[n + i];
      tab[RYS_ASYM_OFF + 2 * (n * (n - 1) / 2 + i)] = (double)(s * s);
      tab[RYS_ASYM_OFF + 2 * (n * (n - 1) / 2 + i) + 1] = (double)w[n + i];
    }
  }
  return tab;
}

}  // namespace

const double* hf_rys_table_host() {
  static std::once_flag once;
  static std::vector<double> tab;
  std::call_once(once, [] { tab = build_rys_table(); });
  return tab.data();
}

extern "C" int hf_rys_rule(int n, double T, double* u, double* w) {
  if (n < 1 || n > RYS_NMAX || !(T >= 0.0) || std::isinf(T) || !u || !w)
    return hf_fail(HF_ERR_INVALID, "hf_rys_rule: n = %d (1..%d), T = %g (finite, >= 0)", n, RYS_NMAX, T);
  const double* tab = hf_rys_table_host();
  for (int i = 0; i < n; ++i) rys_rule_root(tab, n, i, T, u + i, w + i);
  return HF_OK;
}

// ------------------------------------------------------------- device side
namespace hfr {

// Cartesian powers of component c of a shell of angular momentum l (l <= 5),
// packed x | y << 4 | z << 8, at [l (l+1) (l+2) / 6 + c]; order as in the
// basis: x power from l down, then y power from l - x down.
struct CartTable {
  unsigned short v[56];
};
constexpr CartTable make_cart() {
  CartTable t{};
  int k = 0;
  for (int l = 0; l <= 5; ++l)
    for (int x = l; x >= 0; --x)
      for (int y = l - x; y >= 0; --y) t.v[k++] = (unsigned short)(x | (y << 4) | ((l - x - y) << 8));
  return t;
}
__constant__ CartTable kCart = make_cart();

__device__ __forceinline__ int cart(int l, int c) { return kCart.v[l * (l + 1) * (l + 2) / 6 + c]; }

// Fixed part of a warp's shared slice (doubles): transfer coefficients of
// the bra [3][6][6] and the ket, roots, weights, component scales [4][21].
constexpr int kCb = 0, kCd = 108, kRu = 216, kRw = 225, kSc = 240, kHead = 328;

// Outputs of one chunk: at most 32 per lane.
constexpr int kMaxChunk = 1024;

// Work of one class.  The output block (ab|cd) is split into chunks of
// whole rows (a, b) (all c, d), at most kMaxChunk outputs each; a chunk is
// evaluated over the quartet's primitive quartets with its outputs in
// registers (KM per lane).  For the f/g classes every chunk of every
// quartet is its own work item ("native": part = chunk); when HF_JK_RYS
// sends the s/p/d classes here, their lists are split along the primitive
// loop instead and an item walks all chunks.
struct RysClass {
  int la, lb, lc, ld;
  int n;                    // roots
  int na, nb, nc, nd;       // Cartesian components
  int nmax, mmax;           // la + lb, lc + ld
  int SG, SH, SI;           // per-direction sizes of G, bra-transferred H, I
  int oG, oH, oI, oBlk;     // offsets in the warp slice (doubles); the block reuses the tables
  int rpc, nchunks;         // rows (a, b) per chunk, chunks per quartet
  int km;                   // outputs per lane (template of the kernel)
  int native;               // work-item parts are chunks
  int ws;                   // doubles per warp
};

inline RysClass rys_class(int la, int lb, int lc, int ld) {
  RysClass r{};
  r.la = la; r.lb = lb; r.lc = lc; r.ld = ld;
  r.n = (la + lb + lc + ld) / 2 + 1;
  auto nc_ = [](int l) { return (l + 1) * (l + 2) / 2; };
  r.na = nc_(la); r.nb = nc_(lb); r.nc = nc_(lc); r.nd = nc_(ld);
  r.nmax = la + lb;
  r.mmax = lc + ld;
  r.SG = (r.nmax + 1) * (r.mmax + 1);
  r.SH = (la + 1) * (lb + 1) * (r.mmax + 1);
  r.SI = (la + 1) * (lb + 1) * (lc + 1) * (ld + 1);
  r.oG = kHead;
  int end = r.oG + 3 * r.SG;
  r.oH = lb == 0 ? r.oG : end;  // lb = 0: H is G
  if (lb > 0) end = r.oH + 3 * r.SH;
  r.oI = ld == 0 ? r.oH : end;  // ld = 0: I is H
  if (ld > 0) end = r.oI + 3 * r.SI;
  const int ncd = r.nc * r.nd, rows = r.na * r.nb;
  r.rpc = std::max(1, std::min(rows, kMaxChunk / ncd));
  r.nchunks = (rows + r.rpc - 1) / r.rpc;
  const int per_lane = (r.rpc * ncd + 31) / 32;
  r.km = per_lane <= 4 ? 4 : per_lane <= 8 ? 8 : per_lane <= 16 ? 16 : 32;
  r.native = std::max(std::max(la, lb), std::max(lc, ld)) > 2;
  r.oBlk = kHead;
  r.ws = (std::max(end, r.oBlk + r.rpc * ncd) + 1) & ~1;
  return r;
}

// class index -> (la, lb, lc, ld)
inline RysClass rys_class_of(int cls) {
  int X = 0;
  while ((X + 1) * (X + 2) / 2 <= cls) ++X;
  const int Y = cls - X * (X + 1) / 2;
  int la, lb, lc, ld;
  pair_ls(X, &la, &lb);
  pair_ls(Y, &lc, &ld);
  return rys_class(la, lb, lc, ld);
}

__host__ __device__ inline int la1_(const RysClass& rc) { return rc.la + 1; }

// Position (d0, d1, d2, d3) of a flat index in the mixed radix (3, n1, n2,
// n3), d3 fastest, advanced by 32 per step with one carry per digit: the
// transfer loops walk their entries without dividing.
struct Radix {
  int d[4];
  int n[4];
  int s[4];
  __device__ Radix(int e, int n1, int n2, int n3) {
    n[0] = 3; n[1] = n1; n[2] = n2; n[3] = n3;
    d[3] = e % n3; e /= n3;
    d[2] = e % n2; e /= n2;
    d[1] = e % n1; d[0] = e / n1;
    int t = 32;
    s[3] = t % n3; t /= n3;
    s[2] = t % n2; t /= n2;
    s[1] = t % n1; s[0] = t / n1;
  }
  __device__ __forceinline__ void step() {
    int c = 0;
#pragma unroll
    for (int k = 3; k >= 1; --k) {
      d[k] += s[k] + c;
      c = d[k] >= n[k];
      if (c) d[k] -= n[k];
    }
    d[0] += s[0] + c;
  }
};

__device__ __forceinline__ double dfact_odd(int x) {  // (2x-1)!!
  double r = 1.0;
  for (int k = 2 * x - 1; k > 1; k -= 2) r *= k;
  return r;
}

// Per quartet: transfer coefficients C(b,k) AB^(b-k) (bra) and
// C(d,k) CD^(d-k) (ket), and the component scales s(l, c) =
// sqrt((2l-1)!! / ((2x-1)!! (2y-1)!! (2z-1)!!)) of the axial-normalised
// basis.
__device__ void rys_setup(const RysClass& rc, const double* AB, const double* CD, double* s, int lane) {
  for (int e = lane; e < 2 * 108; e += 32) {
    const int side = e / 108, r = e - side * 108;
    const int dir = r / 36, ib = (r / 6) % 6, k = r % 6;
    double v = 0.0;
    if (k <= ib) {
      double bin = 1.0;
      for (int i = 1; i <= k; ++i) bin = bin * (ib - k + i) / i;
      const double x = side ? CD[dir] : AB[dir];
      double pw = 1.0;
      for (int i = 0; i < ib - k; ++i) pw *= x;
      v = bin * pw;
    }
    s[side ? kCd + r : kCb + r] = v;
  }
  for (int e = lane; e < 4 * 21; e += 32) {
    const int sh = e / 21, c = e - sh * 21;
    const int l = sh == 0 ? rc.la : sh == 1 ? rc.lb : sh == 2 ? rc.lc : rc.ld;
    double v = 0.0;
    if (c < (l + 1) * (l + 2) / 2) {
      const int p = cart(l, c);
      v = sqrt(dfact_odd(l) / (dfact_odd(p & 15) * dfact_odd((p >> 4) & 15) * dfact_odd(p >> 8)));
    }
    s[kSc + e] = v;
  }
}

// Rows [r0, r1) of the contracted block of (bra|ket) (row = a NB + b, all
// c, d) over primitive quartets [q_lo, q_hi) (q = bra primitive * ket count
// + ket primitive), written to s + oBlk as [row - r0][c][d], times the
// four component scales.  Only the (ia, ib) rows of the transferred
// tables that the chunk's components use are formed.
template <int KM>
__device__ void rys_rows(const RysClass& rc, const double* __restrict__ prim, const double* __restrict__ rtab,
                         const PairInfo& bra, const PairInfo& ket, int q_lo, int q_hi, int r0, int r1, double* s,
                         int lane) {
  const int NB = rc.nb, NC = rc.nc, ND = rc.nd, NCD = NC * ND;
  const int nout = (r1 - r0) * NCD;
  const int l1 = rc.lb + 1, l3 = rc.ld + 1, ncd_dir = (rc.lc + 1) * (rc.ld + 1);
  // this lane's outputs e = lane + 32 k: offsets into the three I tables
  int idx[KM];
  double acc[KM];
#pragma unroll
  for (int k = 0; k < KM; ++k) {
    acc[k] = 0.0;
    idx[k] = 0;
    const int e = lane + 32 * k;
    if (e < nout) {
      const int rl = e / NCD, cd = e - rl * NCD;
      const int row = r0 + rl, a = row / NB, b = row - a * NB;
      const int c = cd / ND, d = cd - c * ND;
      const int pa = cart(rc.la, a), pb = cart(rc.lb, b), pc = cart(rc.lc, c), pd = cart(rc.ld, d);
      const int ix = ((pa & 15) * l1 + (pb & 15)) * ncd_dir + (pc & 15) * l3 + (pd & 15);
      const int iy = (((pa >> 4) & 15) * l1 + ((pb >> 4) & 15)) * ncd_dir + ((pc >> 4) & 15) * l3 + ((pd >> 4) & 15);
      const int iz = ((pa >> 8) * l1 + (pb >> 8)) * ncd_dir + (pc >> 8) * l3 + (pd >> 8);
      idx[k] = ix | (iy << 10) | (iz << 20);
    }
  }
  // (ia, ib) pairs the chunk needs, per direction (bit ia * (lb+1) + ib)
  unsigned need[3] = {0u, 0u, 0u};
  for (int row = r0 + lane; row < r1; row += 32) {
    const int a = row / NB, b = row - a * NB;
    const int pa = cart(rc.la, a), pb = cart(rc.lb, b);
    need[0] |= 1u << ((pa & 15) * l1 + (pb & 15));
    need[1] |= 1u << (((pa >> 4) & 15) * l1 + ((pb >> 4) & 15));
    need[2] |= 1u << ((pa >> 8) * l1 + (pb >> 8));
  }
#pragma unroll
  for (int d = 0; d < 3; ++d) need[d] = __reduce_or_sync(0xffffffffu, need[d]);
  const int L1 = rc.nmax + 1, M1 = rc.mmax + 1;
  // this lane's first entries of the two transfers, walked 32 at a time
  const Radix hw(lane, la1_(rc), l1, M1), iw(lane, (rc.la + 1) * l1, rc.lc + 1, l3);
  const bool gl = lane < 3 * L1;
  const int gdir = gl ? lane / L1 : 0, gn = gl ? lane - gdir * L1 : 0;
  double* const ru = s + kRu;
  double* const rw = s + kRw;
  const int nk = ket.nprim;
  const double* Ix = s + rc.oI;
  const double* Iy = Ix + rc.SI;
  const double* Iz = Iy + rc.SI;
  __syncwarp();
  for (int qq = q_lo; qq < q_hi; ++qq) {
    const int ib = qq / nk, ik = qq - ib * nk;
    const double* rb = prim + (size_t)(bra.prim0 + ib) * PRIM64_STRIDE;
    const double* rk = prim + (size_t)(ket.prim0 + ik) * PRIM64_STRIDE;
    const double p = __ldg(rb), q = __ldg(rk);
    const double PQx = __ldg(rb + 2) - __ldg(rk + 2), PQy = __ldg(rb + 3) - __ldg(rk + 3),
                 PQz = __ldg(rb + 4) - __ldg(rk + 4);
    const double ipq = 1.0 / (p + q);
    const double T = p * q * ipq * (PQx * PQx + PQy * PQy + PQz * PQz);
    const double pref = __ldg(rb + 8) * __ldg(rk + 8) * sqrt(ipq);
    if (lane < rc.n) rys_rule_root(rtab, rc.n, lane, T, ru + lane, rw + lane);
    const double qf = q * ipq, pf = p * ipq;
    const double PQg = gdir == 0 ? PQx : (gdir == 1 ? PQy : PQz);
    const double PAg = __ldg(rb + 5 + gdir), QCg = __ldg(rk + 5 + gdir);
    const double hp = __ldg(rb + 1), hq = __ldg(rk + 1);  // 1/(2p), 1/(2q)
    __syncwarp();
    for (int r = 0; r < rc.n; ++r) {
      const double u = ru[r];
      const double B00 = 0.5 * u * ipq, B10 = hp * (1.0 - u * qf), B01 = hq * (1.0 - u * pf);
      // G(gn, 0 .. mmax) of direction gdir on this lane
      {
        const double c00 = PAg - u * qf * PQg, d00 = QCg + u * pf * PQg;
        double g = gdir == 2 ? rw[r] * pref : 1.0, gp = 0.0;
        for (int k = 0; k < gn; ++k) {
          const double t = c00 * g + k * B10 * gp;
          gp = g;
          g = t;
        }
        double* Gd = s + rc.oG + gdir * rc.SG + gn * M1;
        if (gl) Gd[0] = g;
        double gm = 0.0;
        for (int m = 0; m < rc.mmax; ++m) {
          const double left = __shfl_up_sync(0xffffffffu, g, 1);  // G(gn - 1, m)
          const double t = d00 * g + m * B01 * gm + (gn > 0 ? gn * B00 * left : 0.0);
          gm = g;
          g = t;
          if (gl) Gd[m + 1] = g;
        }
      }
      __syncwarp();
      if (rc.lb > 0) {  // H(ia, ib, m) = sum_k C(ib,k) AB^(ib-k) G(ia + k, m)
        Radix w = hw;
        for (int e = lane; e < 3 * rc.SH; e += 32, w.step()) {
          const int dir = w.d[0], ia = w.d[1], ib2 = w.d[2], m = w.d[3];
          const unsigned nd = dir == 0 ? need[0] : (dir == 1 ? need[1] : need[2]);
          if (!((nd >> (ia * l1 + ib2)) & 1u)) continue;
          const double* g = s + rc.oG + dir * rc.SG + ia * M1 + m;
          const double* cf = s + kCb + (dir * 6 + ib2) * 6;
          double v = 0.0;
          for (int k = 0; k <= ib2; ++k) v = fma(cf[k], g[k * M1], v);
          s[rc.oH + e] = v;
        }
        __syncwarp();
      }
      if (rc.ld > 0) {  // I(iab, ic, id) = sum_k C(id,k) CD^(id-k) H(iab, ic + k)
        Radix w = iw;
        for (int e = lane; e < 3 * rc.SI; e += 32, w.step()) {
          const int dir = w.d[0], iab = w.d[1], ic = w.d[2], id = w.d[3];
          const unsigned nd = dir == 0 ? need[0] : (dir == 1 ? need[1] : need[2]);
          if (!((nd >> iab) & 1u)) continue;
          const double* h = s + rc.oH + dir * rc.SH + iab * M1 + ic;
          const double* cf = s + kCd + (dir * 6 + id) * 6;
          double v = 0.0;
          for (int k = 0; k <= id; ++k) v = fma(cf[k], h[k], v);
          s[rc.oI + e] = v;
        }
        __syncwarp();
      }
#pragma unroll
      for (int k = 0; k < KM; ++k)
        if (lane + 32 * k < nout) {
          const int t = idx[k];
          acc[k] = fma(Ix[t & 1023] * Iy[(t >> 10) & 1023], Iz[t >> 20], acc[k]);
        }
      __syncwarp();
    }
  }
  // the block overwrites the tables: scale and store
  double* const blk = s + rc.oBlk;
#pragma unroll
  for (int k = 0; k < KM; ++k) {
    const int e = lane + 32 * k;
    if (e < nout) {
      const int rl = e / NCD, cd = e - rl * NCD;
      const int row = r0 + rl, a = row / NB, b = row - a * NB;
      const int c = cd / ND, d = cd - c * ND;
      blk[e] = acc[k] * s[kSc + a] * s[kSc + 21 + b] * s[kSc + 42 + c] * s[kSc + 63 + d];
    }
  }
  __syncwarp();
}

// Work item t -> entry bi, the kets of the item and its part.  Items hold
// w.chunk kets (1 for the Rys classes and the warp-cooperative lists, 32
// for the thread-per-quartet lists).
struct ItemRange {
  int bi, k0, k1, part, nsp;
};
__device__ __forceinline__ void rys_item(const JKWork& w, int t, ItemRange* it) {
  int lo = 0, hi = w.nbra;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(w.ioff + mid) <= t) lo = mid; else hi = mid;
  }
  it->bi = lo;
  it->nsp = w.nsplit ? __ldg(w.nsplit + lo) : 1;
  const int rr = t - __ldg(w.ioff + lo);
  const int blk = rr / it->nsp;
  it->part = rr - blk * it->nsp;
  it->k0 = __ldg(w.kbeg + lo) + blk * w.chunk;
  it->k1 = min(it->k0 + w.chunk, __ldg(w.kend + lo));
}
// Primitive quartets and chunks of one item's part.  Rys lists (nchunk >
// 0): part = range * nchunk + chunk, the range one of nsp / nchunk equal
// slices of the primitive quartets.  Lists built for the Obara-Saika
// kernels (HF_JK_RYS with lists of another shape): every chunk, over a range
// of primitive quartets (chunk 1) or of bra primitive pairs (chunk 32).
__device__ __forceinline__ void rys_part(const RysClass& rc, const JKWork& w, const PairInfo& bra,
                                         const PairInfo& ket, int part, int nsp, int* q_lo, int* q_hi, int* c_lo,
                                         int* c_hi) {
  const int nq = bra.nprim * ket.nprim;
  if (w.nchunk > 0) {
    const int nr = max(1, nsp / w.nchunk), ch = part % w.nchunk, pr = part / w.nchunk;
    *q_lo = pr * nq / nr;
    *q_hi = (pr + 1) * nq / nr;
    *c_lo = ch;
    *c_hi = ch + 1;
  } else {
    *c_lo = 0;
    *c_hi = rc.nchunks;
    if (w.chunk == 1) {
      *q_lo = part * nq / nsp;
      *q_hi = (part + 1) * nq / nsp;
    } else {
      *q_lo = (part * bra.nprim / nsp) * ket.nprim;
      *q_hi = ((part + 1) * bra.nprim / nsp) * ket.nprim;
    }
  }
}

template <int KM>
__global__ void __launch_bounds__(128) rys_jk_kernel(const JKWork w, const PairSet ps, const KernelCommon kc,
                                                     const MolJK one, const MolJK* __restrict__ mols,
                                                     const RysClass rc) {
  extern __shared__ __align__(16) double rsm[];
  double* const s = rsm + (threadIdx.x >> 5) * rc.ws;
  const int lane = threadIdx.x & 31;
  const int NB = rc.nb, NC = rc.nc, ND = rc.nd, NCD = NC * ND;
  for (;;) {
    int t = 0;
    if (lane == 0) t = atomicAdd(w.counter, 1);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= w.nitems) break;
    ItemRange it;
    rys_item(w, t, &it);
    const MolJK* mjp = mols ? mols + __ldg(w.mol + it.bi) : nullptr;
    if (mjp && !mjp->active) continue;
    const PairSet P = mjp ? mjp->ps : ps;
    const int* ketb = mjp ? mjp->ketlist + mjp->ket_off[pair_class(rc.lc, rc.ld)] : w.ket;
    const int bp = __ldg(w.bra + it.bi);
    if (!HF_BCHECK(kc, bp >= 0 && bp < P.npairs, HF_BC_PAIR, bp)) continue;
    const MolJK& mo = mjp ? *mjp : one;
    const int nbf = mo.nbf;
    const PairInfo bra = P.info[bp];
    for (int kidx = it.k0; kidx < it.k1; ++kidx) {
      const int kp = __ldg(ketb + kidx);
      if (!HF_BCHECK(kc, kp >= 0 && kp < P.npairs, HF_BC_PAIR, kp)) continue;
      const PairInfo ket = P.info[kp];
      {
        const bool ok =
            HF_BCHECK(kc, bra.prim0 >= 0 && bra.prim0 + bra.nprim <= P.nprimpairs, HF_BC_PRIM, bra.prim0) &&
            HF_BCHECK(kc, ket.prim0 >= 0 && ket.prim0 + ket.nprim <= P.nprimpairs, HF_BC_PRIM, ket.prim0) &&
            HF_BCHECK(kc, bra.bfA + rc.na <= nbf && bra.bfB + NB <= nbf, HF_BC_MAT, bra.bfA) &&
            HF_BCHECK(kc, ket.bfA + NC <= nbf && ket.bfB + ND <= nbf, HF_BC_MAT, ket.bfA);
        if (!ok) continue;
      }
      int q_lo, q_hi, c_lo, c_hi;
      rys_part(rc, w, bra, ket, it.part, it.nsp, &q_lo, &q_hi, &c_lo, &c_hi);
      if (q_hi <= q_lo) continue;
      rys_setup(rc, bra.AB, ket.AB, s, lane);
      double wdeg = 1.0;
      if (bra.same) wdeg *= 0.5;
      if (ket.same) wdeg *= 0.5;
      if (bp == kp) wdeg *= 0.5;
      const int a0 = bra.bfA, b0 = bra.bfB, c0 = ket.bfA, d0 = ket.bfB;
      const double* __restrict__ Dj = mo.Dj ? mo.Dj : mo.D;
      const int nspin = mo.D2 ? 2 : 1;
      for (int ch = c_lo; ch < c_hi; ++ch) {
        const int r0 = ch * rc.rpc, r1 = min(r0 + rc.rpc, rc.na * NB);
        rys_rows<KM>(rc, P.prim64, kc.rys, bra, ket, q_lo, q_hi, r0, r1, s, lane);
        const double* I = s + rc.oBlk;
        auto Iv = [&](int row, int c, int d) { return I[((row - r0) * NC + c) * ND + d]; };
        auto Dv = [&](const double* Dm, int i, int j) { return __ldg(Dm + (size_t)i * nbf + j); };
        const int af = r0 / NB, al = (r1 - 1) / NB;
        for (int rl = lane; rl < r1 - r0; rl += 32) {  // J'_ab = w sum_cd I D_cd
          const int row = r0 + rl, a = row / NB, b = row - a * NB;
          double v = 0.0;
          for (int c = 0; c < NC; ++c)
            for (int d = 0; d < ND; ++d) v = fma(Iv(row, c, d), Dv(Dj, c0 + c, d0 + d), v);
          hfk::jk_acc(mo.J, (size_t)(a0 + a) * nbf + b0 + b, v * wdeg, kc.det);
        }
        for (int o = lane; o < NCD; o += 32) {  // J'_cd += w sum_(ab in chunk) I D_ab
          const int c = o / ND, d = o % ND;
          double v = 0.0;
          for (int row = r0; row < r1; ++row) {
            const int a = row / NB, b = row - a * NB;
            v = fma(Iv(row, c, d), Dv(Dj, a0 + a, b0 + b), v);
          }
          hfk::jk_acc(mo.J, (size_t)(c0 + c) * nbf + d0 + d, v * wdeg, kc.det);
        }
        for (int sp = 0; sp < nspin; ++sp) {
          const double* __restrict__ Dk = sp ? mo.D2 : mo.D;
          double* __restrict__ Kx = sp ? mo.K2 : mo.K;
          for (int o = lane; o < (al - af + 1) * NC; o += 32) {  // K'_ac += w sum_bd I D_bd
            const int a = af + o / NC, c = o % NC;
            const int bl = max(0, r0 - a * NB), bh = min(NB, r1 - a * NB);
            double v = 0.0;
            for (int b = bl; b < bh; ++b)
              for (int d = 0; d < ND; ++d) v = fma(Iv(a * NB + b, c, d), Dv(Dk, b0 + b, d0 + d), v);
            hfk::jk_acc(Kx, (size_t)(a0 + a) * nbf + c0 + c, v * wdeg, kc.det);
          }
          for (int o = lane; o < (al - af + 1) * ND; o += 32) {  // K'_ad += w sum_bc I D_bc
            const int a = af + o / ND, d = o % ND;
            const int bl = max(0, r0 - a * NB), bh = min(NB, r1 - a * NB);
            double v = 0.0;
            for (int b = bl; b < bh; ++b)
              for (int c = 0; c < NC; ++c) v = fma(Iv(a * NB + b, c, d), Dv(Dk, b0 + b, c0 + c), v);
            hfk::jk_acc(Kx, (size_t)(a0 + a) * nbf + d0 + d, v * wdeg, kc.det);
          }
          for (int o = lane; o < NB * NC; o += 32) {  // K'_bc += w sum_ad I D_ad
            const int b = o / NC, c = o % NC;
            double v = 0.0;
            bool any = false;
            for (int a = af; a <= al; ++a) {
              const int row = a * NB + b;
              if (row < r0 || row >= r1) continue;
              any = true;
              for (int d = 0; d < ND; ++d) v = fma(Iv(row, c, d), Dv(Dk, a0 + a, d0 + d), v);
            }
            if (any) hfk::jk_acc(Kx, (size_t)(b0 + b) * nbf + c0 + c, v * wdeg, kc.det);
          }
          for (int o = lane; o < NB * ND; o += 32) {  // K'_bd += w sum_ac I D_ac
            const int b = o / ND, d = o % ND;
            double v = 0.0;
            bool any = false;
            for (int a = af; a <= al; ++a) {
              const int row = a * NB + b;
              if (row < r0 || row >= r1) continue;
              any = true;
              for (int c = 0; c < NC; ++c) v = fma(Iv(row, c, d), Dv(Dk, a0 + a, c0 + c), v);
            }
            if (any) hfk::jk_acc(Kx, (size_t)(b0 + b) * nbf + d0 + d, v * wdeg, kc.det);
          }
        }
        __syncwarp();
      }
    }
  }
}

// Dense tensor: every element of each quartet's block to its eight index
// permutations (small bases).  An s/p/d item split along its primitive
// loop is taken whole by part 0.
template <int KM>
__global__ void __launch_bounds__(128) rys_store_kernel(const JKWork w, const PairSet ps, const KernelCommon kc,
                                                        double* __restrict__ G, int nbf, const RysClass rc) {
  extern __shared__ __align__(16) double rsm[];
  double* const s = rsm + (threadIdx.x >> 5) * rc.ws;
  const int lane = threadIdx.x & 31;
  const int NB = rc.nb, NC = rc.nc, ND = rc.nd, NCD = NC * ND;
  for (;;) {
    int t = 0;
    if (lane == 0) t = atomicAdd(w.counter, 1);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= w.nitems) break;
    ItemRange it;
    rys_item(w, t, &it);
    // the tensor is written, not accumulated: the first primitive range of
    // each chunk takes the whole primitive loop, the other ranges do nothing
    if (w.nchunk > 0 ? it.part >= w.nchunk : it.part != 0) continue;
    const int bp = __ldg(w.bra + it.bi);
    const PairInfo bra = ps.info[bp];
    for (int kidx = it.k0; kidx < it.k1; ++kidx) {
      const int kp = __ldg(w.ket + kidx);
      const PairInfo ket = ps.info[kp];
      const int c_lo = w.nchunk > 0 ? it.part : 0, c_hi = w.nchunk > 0 ? it.part + 1 : rc.nchunks;
      rys_setup(rc, bra.AB, ket.AB, s, lane);
      for (int ch = c_lo; ch < c_hi; ++ch) {
        const int r0 = ch * rc.rpc, r1 = min(r0 + rc.rpc, rc.na * NB);
        rys_rows<KM>(rc, ps.prim64, kc.rys, bra, ket, 0, bra.nprim * ket.nprim, r0, r1, s, lane);
        const double* I = s + rc.oBlk;
        const size_t n = (size_t)nbf;
        for (int e = lane; e < (r1 - r0) * NCD; e += 32) {
          const int rl = e / NCD, cd = e - rl * NCD;
          const int row = r0 + rl, a = row / NB, b = row - a * NB;
          const int c = cd / ND, d = cd - c * ND;
          const double v = I[e];
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
        __syncwarp();
      }
    }
  }
}

// Q_ab = sqrt(max over components |(ab|ab)|), one warp per pair.
template <int KM>
__global__ void __launch_bounds__(128) rys_schwarz_kernel(const int* __restrict__ pairs, int npairs, const PairSet ps,
                                                          const KernelCommon kc, double* __restrict__ Q,
                                                          const RysClass rc) {
  extern __shared__ __align__(16) double rsm[];
  double* const s = rsm + (threadIdx.x >> 5) * rc.ws;
  const int lane = threadIdx.x & 31;
  const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (t >= npairs) return;
  const int pid = pairs[t];
  const PairInfo pr = ps.info[pid];
  const int NB = rc.nb, NC = rc.nc, ND = rc.nd;
  rys_setup(rc, pr.AB, pr.AB, s, lane);
  double m = 0.0;
  for (int ch = 0; ch < rc.nchunks; ++ch) {
    const int r0 = ch * rc.rpc, r1 = min(r0 + rc.rpc, rc.na * NB);
    rys_rows<KM>(rc, ps.prim64, kc.rys, pr, pr, 0, pr.nprim * pr.nprim, r0, r1, s, lane);
    const double* I = s + rc.oBlk;
    for (int row = r0 + lane; row < r1; row += 32) {
      const int a = row / NB, b = row - a * NB;
      m = fmax(m, fabs(I[((row - r0) * NC + a) * ND + b]));
    }
    __syncwarp();
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) Q[pid] = sqrt(m);
}

// ------------------------------------------------------------- nuclear gradient
// Derivative integrals for the analytic RHF gradient.  A primitive's
// derivative with respect to its centre is d/dA_x [x_A^a e^(-alpha x_A^2)]
// = 2 alpha x_A^(a+1) e - a x_A^(a-1) e, so per direction the one-dimensional
// factor of (ab|cd) with respect to A becomes 2 alpha I(a+1, b, c, d) -
// a I(a-1, b, c, d) (likewise b, beta for B and c, gamma for C); D follows
// by translational invariance, dD = -(dA + dB + dC).  The tables are one
// power higher on A, B and C than the energy's.  Each warp contracts its
// quartet's derivative integrals on the fly with
//     Gamma = 8 w [2 D_ab D_cd - (D_ac D_bd + D_ad D_bc) / 2]
// (w the symmetry weight of the unique quartet), the two-electron part of
// dE/dR = sum over unique quartets of Gamma d(ab|cd)/dR with the energy
// E_2e = 2 Tr[D J] - Tr[D K].
struct GradClass {
  RysClass base;        // the J/K class: chunks and work-list shape
  int n;                // roots (total angular momentum + 1)
  int NG, MG;           // highest G powers: la + lb + 1, lc + ld + 1
  int SG, SH, SI;       // per-direction table sizes
  int oG, oH, oI, oX;   // offsets in the warp slice (doubles); oX: per-output table
  int ws;
};

inline GradClass grad_class(const RysClass& rc) {
  GradClass g{};
  g.base = rc;
  g.n = (rc.la + rc.lb + rc.lc + rc.ld + 1) / 2 + 1;
  g.NG = rc.nmax + 1;
  g.MG = rc.mmax + 1;
  g.SG = (g.NG + 1) * (g.MG + 1);
  g.SH = (rc.la + 2) * (rc.lb + 2) * (g.MG + 1);
  g.SI = (rc.la + 2) * (rc.lb + 2) * (rc.lc + 2) * (rc.ld + 1);
  g.oG = kHead;
  g.oH = g.oG + 3 * g.SG;
  int end = g.oH + 3 * g.SH;
  g.oI = rc.ld == 0 ? g.oH : end;  // ld = 0: I is H (ic = m)
  if (rc.ld > 0) end = g.oI + 3 * g.SI;
  g.oX = (end + 1) & ~1;
  g.ws = g.oX + 3 * rc.rpc * rc.nc * rc.nd;
  g.ws = (g.ws + 1) & ~1;
  return g;
}

__global__ void __launch_bounds__(128) rys_grad_kernel(const JKWork w, const PairSet ps, const KernelCommon kc,
                                                       const double* __restrict__ D,
                                                       const int* __restrict__ bf_atom, int nbf,
                                                       double* __restrict__ grad, const GradClass gc) {
  extern __shared__ __align__(16) double rsm[];
  const RysClass& rc = gc.base;
  double* const s = rsm + (threadIdx.x >> 5) * gc.ws;
  const int lane = threadIdx.x & 31;
  const int NB = rc.nb, NC = rc.nc, ND = rc.nd, NCD = NC * ND;
  const int lb2 = rc.lb + 2, lc2 = rc.lc + 2, ld1 = rc.ld + 1;
  const int sC = ld1, sB = lc2 * ld1, sA = lb2 * lc2 * ld1;
  const int L1 = gc.NG + 1, M1 = gc.MG + 1;
  const bool gl = lane < 3 * L1;
  const int gdir = gl ? lane / L1 : 0, gn = gl ? lane - gdir * L1 : 0;
  double* const ru = s + kRu;
  double* const rw = s + kRw;
  for (;;) {
    int t = 0;
    if (lane == 0) t = atomicAdd(w.counter, 1);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= w.nitems) break;
    ItemRange it;
    rys_item(w, t, &it);
    const int bp = __ldg(w.bra + it.bi);
    if (!HF_BCHECK(kc, bp >= 0 && bp < ps.npairs, HF_BC_PAIR, bp)) continue;
    const PairInfo bra = ps.info[bp];
    for (int kidx = it.k0; kidx < it.k1; ++kidx) {
      const int kp = __ldg(w.ket + kidx);
      if (!HF_BCHECK(kc, kp >= 0 && kp < ps.npairs, HF_BC_PAIR, kp)) continue;
      const PairInfo ket = ps.info[kp];
      int q_lo, q_hi, c_lo, c_hi;
      rys_part(rc, w, bra, ket, it.part, it.nsp, &q_lo, &q_hi, &c_lo, &c_hi);
      if (q_hi <= q_lo) continue;
      rys_setup(rc, bra.AB, ket.AB, s, lane);
      double wdeg = 8.0;
      if (bra.same) wdeg *= 0.5;
      if (ket.same) wdeg *= 0.5;
      if (bp == kp) wdeg *= 0.5;
      const int a0 = bra.bfA, b0 = bra.bfB, c0 = ket.bfA, d0 = ket.bfB;
      double g[9];  // dE/dA, dE/dB, dE/dC (x, y, z each)
#pragma unroll
      for (int k = 0; k < 9; ++k) g[k] = 0.0;
      for (int ch = c_lo; ch < c_hi; ++ch) {
        const int r0 = ch * rc.rpc, r1 = min(r0 + rc.rpc, rc.na * NB);
        const int nout = (r1 - r0) * NCD;
        __syncwarp();
        // per output: Gamma (scaled), table offsets, Cartesian powers
        double* X = s + gc.oX;
        for (int e = lane; e < nout; e += 32) {
          const int rl = e / NCD, cd = e - rl * NCD;
          const int row = r0 + rl, a = row / NB, b = row - a * NB;
          const int c = cd / ND, d = cd - c * ND;
          const int pa = cart(rc.la, a), pb = cart(rc.lb, b), pc = cart(rc.lc, c), pd = cart(rc.ld, d);
          auto off = [&](int sh) {
            return ((((pa >> sh) & 15) * lb2 + ((pb >> sh) & 15)) * lc2 + ((pc >> sh) & 15)) * ld1 + ((pd >> sh) & 15);
          };
          auto Dv = [&](int i, int j) { return __ldg(D + (size_t)i * nbf + j); };
          const int ia = a0 + a, ib = b0 + b, ic = c0 + c, id = d0 + d;
          const double gam = wdeg * s[kSc + a] * s[kSc + 21 + b] * s[kSc + 42 + c] * s[kSc + 63 + d] *
                             (2.0 * Dv(ia, ib) * Dv(ic, id) - 0.5 * (Dv(ia, ic) * Dv(ib, id) + Dv(ia, id) * Dv(ib, ic)));
          const long long idx = (long long)off(0) | ((long long)off(4) << 21) | ((long long)off(8) << 42);
          const long long pw = (long long)(pa & 0xfff) | ((long long)(pb & 0xfff) << 12) | ((long long)(pc & 0xfff) << 24);
          X[3 * e] = gam;
          X[3 * e + 1] = __longlong_as_double(idx);
          X[3 * e + 2] = __longlong_as_double(pw);
        }
        __syncwarp();
        const int nk = ket.nprim;
        for (int qq = q_lo; qq < q_hi; ++qq) {
          const int ibp = qq / nk, ikp = qq - ibp * nk;
          const double* rb = ps.prim64 + (size_t)(bra.prim0 + ibp) * PRIM64_STRIDE;
          const double* rk = ps.prim64 + (size_t)(ket.prim0 + ikp) * PRIM64_STRIDE;
          const double p = __ldg(rb), q = __ldg(rk);
          const double PQx = __ldg(rb + 2) - __ldg(rk + 2), PQy = __ldg(rb + 3) - __ldg(rk + 3),
                       PQz = __ldg(rb + 4) - __ldg(rk + 4);
          const double ipq = 1.0 / (p + q);
          const double T = p * q * ipq * (PQx * PQx + PQy * PQy + PQz * PQz);
          const double pref = __ldg(rb + 8) * __ldg(rk + 8) * sqrt(ipq);
          const double za2 = 2.0 * __ldg(rb + 9), zb2 = 2.0 * (p - __ldg(rb + 9)), zc2 = 2.0 * __ldg(rk + 9);
          if (lane < gc.n) rys_rule_root(kc.rys, gc.n, lane, T, ru + lane, rw + lane);
          const double qf = q * ipq, pf = p * ipq;
          const double PQg = gdir == 0 ? PQx : (gdir == 1 ? PQy : PQz);
          const double PAg = __ldg(rb + 5 + gdir), QCg = __ldg(rk + 5 + gdir);
          const double hp = __ldg(rb + 1), hq = __ldg(rk + 1);
          __syncwarp();
          for (int r = 0; r < gc.n; ++r) {
            const double u = ru[r];
            const double B00 = 0.5 * u * ipq, B10 = hp * (1.0 - u * qf), B01 = hq * (1.0 - u * pf);
            {
              const double c00 = PAg - u * qf * PQg, d00 = QCg + u * pf * PQg;
              double gg = gdir == 2 ? rw[r] * pref : 1.0, gp = 0.0;
              for (int k = 0; k < gn; ++k) {
                const double tt = c00 * gg + k * B10 * gp;
                gp = gg;
                gg = tt;
              }
              double* Gd = s + gc.oG + gdir * gc.SG + gn * M1;
              if (gl) Gd[0] = gg;
              double gm = 0.0;
              for (int m = 0; m < gc.MG; ++m) {
                const double left = __shfl_up_sync(0xffffffffu, gg, 1);
                const double tt = d00 * gg + m * B01 * gm + (gn > 0 ? gn * B00 * left : 0.0);
                gm = gg;
                gg = tt;
                if (gl) Gd[m + 1] = gg;
              }
            }
            __syncwarp();
            {  // H(ia, ib, m), ia <= la + 1, ib <= lb + 1
              Radix wk(lane, rc.la + 2, lb2, M1);
              for (int e = lane; e < 3 * gc.SH; e += 32, wk.step()) {
                const int dir = wk.d[0], ia = wk.d[1], ib2 = wk.d[2], m = wk.d[3];
                const double* gp2 = s + gc.oG + dir * gc.SG + ia * M1 + m;
                const double* cf = s + kCb + (dir * 6 + ib2) * 6;
                double v = 0.0;
                if (ia + ib2 <= gc.NG)
                  for (int k = 0; k <= ib2; ++k) v = fma(cf[k], gp2[k * M1], v);
                s[gc.oH + e] = v;
              }
              __syncwarp();
            }
            if (rc.ld > 0) {  // I(iab, ic, id), ic <= lc + 1, id <= ld
              Radix wk(lane, (rc.la + 2) * lb2, lc2, ld1);
              for (int e = lane; e < 3 * gc.SI; e += 32, wk.step()) {
                const int dir = wk.d[0], iab = wk.d[1], ic = wk.d[2], id = wk.d[3];
                const double* h = s + gc.oH + dir * gc.SH + iab * M1 + ic;
                const double* cf = s + kCd + (dir * 6 + id) * 6;
                double v = 0.0;
                if (ic + id <= gc.MG)
                  for (int k = 0; k <= id; ++k) v = fma(cf[k], h[k], v);
                s[gc.oI + e] = v;
              }
              __syncwarp();
            }
            const double* Ix = s + gc.oI;
            const double* Iy = Ix + gc.SI;
            const double* Iz = Iy + gc.SI;
            for (int e = lane; e < nout; e += 32) {
              const double gam = X[3 * e];
              const long long idx = __double_as_longlong(X[3 * e + 1]);
              const long long pw = __double_as_longlong(X[3 * e + 2]);
              const int o3[3] = {(int)(idx & 0x1fffff), (int)((idx >> 21) & 0x1fffff), (int)(idx >> 42)};
              const double* I3[3] = {Ix, Iy, Iz};
              double v0[3], vA[3], vB[3], vC[3];
#pragma unroll
              for (int dd = 0; dd < 3; ++dd) {
                const double* Id = I3[dd];
                const int o = o3[dd];
                const int na_ = (int)((pw >> (4 * dd)) & 15), nb_ = (int)((pw >> (12 + 4 * dd)) & 15),
                          nc_ = (int)((pw >> (24 + 4 * dd)) & 15);
                v0[dd] = Id[o];
                vA[dd] = za2 * Id[o + sA] - (na_ > 0 ? na_ * Id[o - sA] : 0.0);
                vB[dd] = zb2 * Id[o + sB] - (nb_ > 0 ? nb_ * Id[o - sB] : 0.0);
                vC[dd] = zc2 * Id[o + sC] - (nc_ > 0 ? nc_ * Id[o - sC] : 0.0);
              }
              const double yz = v0[1] * v0[2], xz = v0[0] * v0[2], xy = v0[0] * v0[1];
              g[0] = fma(gam, vA[0] * yz, g[0]);
              g[1] = fma(gam, vA[1] * xz, g[1]);
              g[2] = fma(gam, vA[2] * xy, g[2]);
              g[3] = fma(gam, vB[0] * yz, g[3]);
              g[4] = fma(gam, vB[1] * xz, g[4]);
              g[5] = fma(gam, vB[2] * xy, g[5]);
              g[6] = fma(gam, vC[0] * yz, g[6]);
              g[7] = fma(gam, vC[1] * xz, g[7]);
              g[8] = fma(gam, vC[2] * xy, g[8]);
            }
            __syncwarp();
          }
        }
      }
#pragma unroll
      for (int k = 0; k < 9; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) g[k] += __shfl_xor_sync(0xffffffffu, g[k], o);
      if (lane == 0) {
        const int at[3] = {__ldg(bf_atom + a0), __ldg(bf_atom + b0), __ldg(bf_atom + c0)};
        const int atD = __ldg(bf_atom + d0);
#pragma unroll
        for (int x = 0; x < 3; ++x) {
          atomicAdd(grad + 3 * at[0] + x, g[x]);
          atomicAdd(grad + 3 * at[1] + x, g[3 + x]);
          atomicAdd(grad + 3 * at[2] + x, g[6 + x]);
          atomicAdd(grad + 3 * atD + x, -(g[x] + g[3 + x] + g[6 + x]));
        }
      }
    }
  }
}

// ------------------------------------------------------------- launchers
size_t smem_of(const RysClass& rc, int warps) { return (size_t)warps * rc.ws * sizeof(double); }

template <int KM>
void set_smem_attr_km() {
  static std::once_flag once;
  std::call_once(once, [] {
    const int mx = 227 * 1024;
    cudaFuncSetAttribute(rys_jk_kernel<KM>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(rys_store_kernel<KM>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(rys_schwarz_kernel<KM>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  });
}

// dispatch on the class's outputs per lane
#define RYS_KM_DISPATCH(rc, F)   \
  switch ((rc).km) {             \
    case 4: F(4); break;         \
    case 8: F(8); break;         \
    case 16: F(16); break;       \
    default: F(32); break;       \
  }

template <int CLS>
void jk_launch(const JKWork& w, const PairSet& ps, const KernelCommon& kc, const MolJK& one, const MolJK* mols,
               int grid, int threads, cudaStream_t st) {
  static const RysClass rc = rys_class_of(CLS);
#define RYS_L(KM)          \
  set_smem_attr_km<KM>(); \
  rys_jk_kernel<KM><<<grid, threads, smem_of(rc, threads / 32), st>>>(w, ps, kc, one, mols, rc)
  RYS_KM_DISPATCH(rc, RYS_L)
#undef RYS_L
}

template <int CLS>
int jk_occ() {
  static const RysClass rc = rys_class_of(CLS);
  int n = 0;
#define RYS_O(KM)          \
  set_smem_attr_km<KM>(); \
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, rys_jk_kernel<KM>, 128, smem_of(rc, 4))
  RYS_KM_DISPATCH(rc, RYS_O)
#undef RYS_O
  return n;
}

template <int CLS>
void store_launch(const JKWork& w, const PairSet& ps, const KernelCommon& kc, double* G, int nbf, int grid,
                  cudaStream_t st) {
  static const RysClass rc = rys_class_of(CLS);
#define RYS_S(KM)          \
  set_smem_attr_km<KM>(); \
  rys_store_kernel<KM><<<grid, 128, smem_of(rc, 4), st>>>(w, ps, kc, G, nbf, rc)
  RYS_KM_DISPATCH(rc, RYS_S)
#undef RYS_S
}

template <int CLS>
void schwarz_launch(const int* pairs, int npairs, const PairSet& ps, const KernelCommon& kc, double* Q,
                    cudaStream_t st) {
  if (npairs <= 0) return;
  static const RysClass rc = rys_class_of(CLS);
#define RYS_Q(KM)          \
  set_smem_attr_km<KM>(); \
  rys_schwarz_kernel<KM><<<(npairs + 3) / 4, 128, smem_of(rc, 4), st>>>(pairs, npairs, ps, kc, Q, rc)
  RYS_KM_DISPATCH(rc, RYS_Q)
#undef RYS_Q
}

template <int CLS>
void grad_launch(const JKWork& w, const PairSet& ps, const KernelCommon& kc, const double* D, const int* bf_atom,
                 int nbf, double* grad, int grid, cudaStream_t st) {
  static const GradClass gc = grad_class(rys_class_of(CLS));
  static std::once_flag once;
  std::call_once(once, [] {
    cudaFuncSetAttribute(rys_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  });
  // four warps per block where their slices fit in 227 KB, else two
  const int warps = 4 * gc.ws * (int)sizeof(double) <= 227 * 1024 ? 4 : 2;
  const int blocks = std::max(1, std::min(grid, (w.nitems + warps - 1) / warps));
  rys_grad_kernel<<<blocks, 32 * warps, (size_t)warps * gc.ws * sizeof(double), st>>>(w, ps, kc, D, bf_atom, nbf,
                                                                                       grad, gc);
}

template <size_t... I>
void register_all(EriClassOps* table, std::index_sequence<I...>) {
  static const char* const kL = "spdfg";
  static char names[HF_NCLASS][16];
  const jk_launch_fn jk[] = {&jk_launch<(int)I>...};
  const occ_fn occ[] = {&jk_occ<(int)I>...};
  const store_launch_fn store[] = {&store_launch<(int)I>...};
  const schwarz_launch_fn schw[] = {&schwarz_launch<(int)I>...};
  const grad_launch_fn grd[] = {&grad_launch<(int)I>...};
  jk_launch_fn jkt[HF_NCLASS] = {};
  occ_fn occt[HF_NCLASS] = {};
  ::hf_rys_thread_classes(jkt, occt);
  for (int c = 0; c < HF_NCLASS; ++c) {
    EriClassOps& e = table[c];
    e.jkrys = jk[c];
    e.occrys = occ[c];
    e.grad = grd[c];
    const RysClass rc = rys_class_of(c);
    e.rys_nchunks = rc.nchunks;
    e.rys_native = rc.native;
    if (!rc.native) continue;  // Obara-Saika classes
    // f/g classes: the Rys kernel in every precision mode (FP64 arithmetic);
    // each work item is one chunk of one quartet
    e.jk64 = e.jk32 = e.jkdf = jk[c];
    e.occ64 = e.occ32 = e.occdf = occ[c];
    e.store = store[c];
    e.schwarz = schw[c];
    e.chunk = 1;
    if (jkt[c]) {  // small f/g class: 32 kets per item, one per lane
      e.jk64 = e.jk32 = e.jkdf = jkt[c];
      e.occ64 = e.occ32 = e.occdf = occt[c];
      e.chunk = 32;
    }
    // operation count per primitive quartet (an FMA counts 2): set-up, the
    // rule (two Clenshaw sums per root), then per root the G recurrences,
    // both transfers and the Ix Iy Iz products into the block; per
    // contracted quartet the component scaling.  Chunks that repeat the
    // recurrences are not counted.
    const int nabcd = rc.na * rc.nb * rc.nc * rc.nd, M1 = rc.mmax + 1;
    int per_root = 3 * rc.SG * 5 + 3 * nabcd;
    if (rc.lb > 0) per_root += 3 * (rc.la + 1) * M1 * ((rc.lb + 1) * (rc.lb + 2) / 2) * 2;
    if (rc.ld > 0) per_root += 3 * (rc.la + 1) * (rc.lb + 1) * (rc.lc + 1) * ((rc.ld + 1) * (rc.ld + 2) / 2) * 2;
    e.vrr_flops = 30 + rc.n * (4 * RYS_NCHEB + 10) + rc.n * per_root;
    e.hrr_flops = nabcd;
    snprintf(names[c], sizeof(names[c]), "R_%c%c_%c%c", kL[rc.la], kL[rc.lb], kL[rc.lc], kL[rc.ld]);
    e.name = names[c];
  }
}

}  // namespace hfr

void hf_register_classes_rys(EriClassOps* table) {
  hfr::register_all(table, std::make_index_sequence<HF_NCLASS>{});
}
