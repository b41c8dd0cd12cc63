// onee.cu -- one-electron matrices S, T, V of Eqs. 2-4 by the Obara-Saika
// recurrences (setup work, O(nbf^2) per molecule).
//
//   overlap, per axis:  S_{i+1,j} = PA S_ij + (i S_{i-1,j} + j S_{i,j-1}) / (2p)
//                       S_{i,j+1} = PB S_ij + (i S_{i-1,j} + j S_{i,j-1}) / (2p)
//                       S_00 = sqrt(pi/p) exp(-ab/p AB_x^2)
//   kinetic, per axis (Laplacian on the ket):
//                       T_ij = -1/2 [ j(j-1) S_{i,j-2} - 2b(2j+1) S_ij + 4b^2 S_{i,j+2} ]
//                       T = Tx Sy Sz + Sx Ty Sz + Sx Sy Tz
//   nuclear attraction (auxiliary index m, nucleus C):
//                       Th(e+1_i)^(m) = PA_i Th(e)^(m) - PC_i Th(e)^(m+1)
//                                       + e_i/(2p) (Th(e-1_i)^(m) - Th(e-1_i)^(m+1))
//                       Th(0)^(m) = 2 pi / p exp(-ab/p |AB|^2) F_m(p |PC|^2)
//                       (a|b) from Th(a+k) by the binomial transfer
//                       (x-B)^b = sum_k C(b,k) (x-A)^k (A-B)^(b-k).
//   for la + lb > 4 (f and g shells) the nuclear attraction is taken by Rys
//   quadrature instead: with n = (la+lb)/2 + 1 roots u of the rule at
//   T = p |PC|^2, (a|1/r_C|b) = 2 pi / p exp(-ab/p |AB|^2)
//   sum_u w_u Ix Iy Iz, the one-dimensional factors from
//                       I(i+1) = (PA - u PC) I(i) + i (1 - u) / (2p) I(i-1),
//                       I(0) = 1, and the same transfer to B.
#include <cmath>

#include "eri.cuh"
#include "hf_internal.h"
#include "rys.cuh"

namespace {

__device__ __forceinline__ void cart_pow(int l, int c, int* p) {
  int k = 0;
  for (int x = l; x >= 0; --x)
    for (int y = l - x; y >= 0; --y) {
      if (k == c) { p[0] = x; p[1] = y; p[2] = l - x - y; return; }
      ++k;
    }
}

// scale of Cartesian component c of an axial-normalised shell of angular
// momentum l: sqrt((2l-1)!! / ((2x-1)!! (2y-1)!! (2z-1)!!))
__device__ double comp_scale_any(int l, int c) {
  int p[3];
  cart_pow(l, c, p);
  auto df = [](int x) {
    double r = 1.0;
    for (int k = 2 * x - 1; k > 1; k -= 2) r *= k;
    return r;
  };
  return sqrt(df(l) / (df(p[0]) * df(p[1]) * df(p[2])));
}

__device__ double binom(int n, int k) {
  double r = 1.0;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return r;
}

__device__ void boys_any(int L, double T, const double* tab, double* F) {
  switch (L) {
    case 0: hfk::boys64<0>(T, tab, F); break;
    case 1: hfk::boys64<1>(T, tab, F); break;
    case 2: hfk::boys64<2>(T, tab, F); break;
    case 3: hfk::boys64<3>(T, tab, F); break;
    default: hfk::boys64<4>(T, tab, F); break;
  }
}

// thread per (i, j) basis-function pair
__global__ void one_electron_kernel(int nbf, const int* __restrict__ bf_shell, const int* __restrict__ sh_l,
                                    const int* __restrict__ sh_bf, const int* __restrict__ sh_nprim,
                                    const int* __restrict__ sh_prim, const double* __restrict__ sh_xyz,
                                    const double* __restrict__ exps, const double* __restrict__ coefs, int natom,
                                    const double* __restrict__ atom_xyz, const int* __restrict__ atom_Z,
                                    const double* __restrict__ boys, const double* __restrict__ rys,
                                    double* __restrict__ S, double* __restrict__ T, double* __restrict__ V) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)nbf * nbf) return;
  const int i = (int)(t / nbf), j = (int)(t % nbf);
  const int sa = bf_shell[i], sb = bf_shell[j];
  const int la = sh_l[sa], lb = sh_l[sb];
  int pa[3], pb[3];
  cart_pow(la, i - sh_bf[sa], pa);
  cart_pow(lb, j - sh_bf[sb], pb);
  const double* A = sh_xyz + 3 * sa;
  const double* B = sh_xyz + 3 * sb;
  const double scale = comp_scale_any(la, i - sh_bf[sa]) * comp_scale_any(lb, j - sh_bf[sb]);
  double AB[3], r2 = 0.0;
  for (int x = 0; x < 3; ++x) {
    AB[x] = A[x] - B[x];
    r2 += AB[x] * AB[x];
  }
  double s_sum = 0.0, t_sum = 0.0, v_sum = 0.0;
  for (int ka = 0; ka < sh_nprim[sa]; ++ka)
    for (int kb = 0; kb < sh_nprim[sb]; ++kb) {
      const double a = exps[sh_prim[sa] + ka], b = exps[sh_prim[sb] + kb];
      const double c = coefs[sh_prim[sa] + ka] * coefs[sh_prim[sb] + kb];
      const double p = a + b, o2p = 0.5 / p, mu = a * b / p;
      double P[3], PA[3], PB[3];
      for (int x = 0; x < 3; ++x) {
        P[x] = (a * A[x] + b * B[x]) / p;
        PA[x] = P[x] - A[x];
        PB[x] = P[x] - B[x];
      }
      // 1D overlaps S[x][i][j], i <= la, j <= lb + 2
      double S1[3][5][7];
      for (int x = 0; x < 3; ++x) {
        double (*s)[7] = S1[x];
        s[0][0] = sqrt(3.14159265358979323846 / p) * exp(-mu * AB[x] * AB[x]);
        for (int ii = 0; ii < pa[x]; ++ii) s[ii + 1][0] = PA[x] * s[ii][0] + (ii > 0 ? ii * o2p * s[ii - 1][0] : 0.0);
        for (int ii = 0; ii <= pa[x]; ++ii)
          for (int jj = 0; jj < pb[x] + 2; ++jj)
            s[ii][jj + 1] = PB[x] * s[ii][jj] + ((ii > 0 ? ii * s[ii - 1][jj] : 0.0) + (jj > 0 ? jj * s[ii][jj - 1] : 0.0)) * o2p;
      }
      const double sx = S1[0][pa[0]][pb[0]], sy = S1[1][pa[1]][pb[1]], sz = S1[2][pa[2]][pb[2]];
      double tk[3];
      for (int x = 0; x < 3; ++x) {
        const int jj = pb[x];
        double v = -2.0 * b * (2 * jj + 1) * S1[x][pa[x]][jj] + 4.0 * b * b * S1[x][pa[x]][jj + 2];
        if (jj >= 2) v += jj * (jj - 1) * S1[x][pa[x]][jj - 2];
        tk[x] = -0.5 * v;
      }
      s_sum += c * sx * sy * sz;
      t_sum += c * (tk[0] * sy * sz + sx * tk[1] * sz + sx * sy * tk[2]);
      // nuclear attraction
      const int L = la + lb;
      const double pre = 2.0 * 3.14159265358979323846 / p * exp(-mu * r2);
      for (int at = 0; at < natom; ++at) {
        if (atom_Z[at] == 0) continue;
        const double* Cc = atom_xyz + 3 * at;
        double PC[3] = {P[0] - Cc[0], P[1] - Cc[1], P[2] - Cc[2]};
        if (L > 4) {  // Rys quadrature
          const int nr = L / 2 + 1;
          const double Tn = p * (PC[0] * PC[0] + PC[1] * PC[1] + PC[2] * PC[2]);
          double vr = 0.0;
          for (int r = 0; r < nr; ++r) {
            double u, w;
            rys_rule_root(rys, nr, r, Tn, &u, &w);
            double prod = w;
            for (int x = 0; x < 3; ++x) {
              double g[9];
              g[0] = 1.0;
              const double c00 = PA[x] - u * PC[x], b10 = (1.0 - u) * o2p;
              for (int k = 0; k < pa[x] + pb[x]; ++k) g[k + 1] = c00 * g[k] + (k > 0 ? k * b10 * g[k - 1] : 0.0);
              double v = 0.0;
              for (int k = 0; k <= pb[x]; ++k) v += binom(pb[x], k) * pow(AB[x], pb[x] - k) * g[pa[x] + k];
              prod *= v;
            }
            vr += prod;
          }
          v_sum -= c * atom_Z[at] * pre * vr;
          continue;
        }
        double F[5];
        boys_any(L, p * (PC[0] * PC[0] + PC[1] * PC[1] + PC[2] * PC[2]), boys, F);
        // Th[ex][ey][ez][m], total l <= 4
        double Th[5][5][5][5];
        for (int m = 0; m <= L; ++m) Th[0][0][0][m] = pre * F[m];
        for (int tot = 1; tot <= L; ++tot)
          for (int ex = tot; ex >= 0; --ex)
            for (int ey = tot - ex; ey >= 0; --ey) {
              const int ez = tot - ex - ey;
              const int e[3] = {ex, ey, ez};
              int ax = 0;
              if (e[1] > e[ax]) ax = 1;
              if (e[2] > e[ax]) ax = 2;
              int f[3] = {ex, ey, ez};
              f[ax] -= 1;
              for (int m = 0; m <= L - tot; ++m) {
                double v = PA[ax] * Th[f[0]][f[1]][f[2]][m] - PC[ax] * Th[f[0]][f[1]][f[2]][m + 1];
                if (f[ax] > 0) {
                  int g[3] = {f[0], f[1], f[2]};
                  g[ax] -= 1;
                  v += f[ax] * o2p * (Th[g[0]][g[1]][g[2]][m] - Th[g[0]][g[1]][g[2]][m + 1]);
                }
                Th[ex][ey][ez][m] = v;
              }
            }
        double vab = 0.0;
        for (int kx = 0; kx <= pb[0]; ++kx)
          for (int ky = 0; ky <= pb[1]; ++ky)
            for (int kz = 0; kz <= pb[2]; ++kz) {
              const double w = binom(pb[0], kx) * binom(pb[1], ky) * binom(pb[2], kz) * pow(AB[0], pb[0] - kx) *
                               pow(AB[1], pb[1] - ky) * pow(AB[2], pb[2] - kz);
              vab += w * Th[pa[0] + kx][pa[1] + ky][pa[2] + kz][0];
            }
        v_sum -= c * atom_Z[at] * vab;
      }
    }
  S[t] = s_sum * scale;
  T[t] = t_sum * scale;
  V[t] = v_sum * scale;
}

}  // namespace

int hf_basis_one_electron(hf_basis* b) {
  if (b->have_one) return HF_OK;
  hf_ctx* ctx = b->ctx;
  cudaStream_t st = ctx->stream;
  const int n = b->nbf, ns = b->nshell;
  std::vector<int> bf_shell(n);
  for (int s = 0; s < ns; ++s)
    for (int k = b->sh_bf[s]; k < b->sh_bf[s + 1]; ++k) bf_shell[k] = s;
  std::vector<double> sh_xyz(3 * ns), at_xyz(3 * b->natom);
  std::vector<int> Z(b->natom);
  for (int s = 0; s < ns; ++s)
    for (int x = 0; x < 3; ++x) sh_xyz[3 * s + x] = b->atoms[b->sh_atom[s]].xyz[x];
  for (int a = 0; a < b->natom; ++a) {
    Z[a] = b->atoms[a].Z;
    for (int x = 0; x < 3; ++x) at_xyz[3 * a + x] = b->atoms[a].xyz[x];
  }
  DevArray<int> dbs, dl, dbf, dn, dp, dZ;
  DevArray<double> dsx, dex, dco, dax;
  HF_CHECK(dbs.alloc(ctx, n));
  HF_CHECK(dl.alloc(ctx, ns));
  HF_CHECK(dbf.alloc(ctx, ns + 1));
  HF_CHECK(dn.alloc(ctx, ns));
  HF_CHECK(dp.alloc(ctx, ns));
  HF_CHECK(dZ.alloc(ctx, b->natom));
  HF_CHECK(dsx.alloc(ctx, 3 * ns));
  HF_CHECK(dex.alloc(ctx, b->nprim));
  HF_CHECK(dco.alloc(ctx, b->nprim));
  HF_CHECK(dax.alloc(ctx, 3 * b->natom));
  HF_CHECK(b->S.alloc(ctx, (size_t)n * n));
  HF_CHECK(b->T.alloc(ctx, (size_t)n * n));
  HF_CHECK(b->V.alloc(ctx, (size_t)n * n));
  HF_CUDA(cudaMemcpyAsync(dbs.ptr, bf_shell.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st));
  HF_CUDA(cudaMemcpyAsync(dl.ptr, b->sh_l.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, st));
  HF_CUDA(cudaMemcpyAsync(dbf.ptr, b->sh_bf.data(), sizeof(int) * (ns + 1), cudaMemcpyHostToDevice, st));
  HF_CUDA(cudaMemcpyAsync(dn.ptr, b->sh_nprim.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, st));
  HF_CUDA(cudaMemcpyAsync(dp.ptr, b->sh_prim.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, st));
  HF_CUDA(cudaMemcpyAsync(dZ.ptr, Z.data(), sizeof(int) * b->natom, cudaMemcpyHostToDevice, st));
  HF_CUDA(cudaMemcpyAsync(dsx.ptr, sh_xyz.data(), sizeof(double) * 3 * ns, cudaMemcpyHostToDevice, st));
  HF_CUDA(cudaMemcpyAsync(dex.ptr, b->exps.data(), sizeof(double) * b->nprim, cudaMemcpyHostToDevice, st));
  HF_CUDA(cudaMemcpyAsync(dco.ptr, b->coefs.data(), sizeof(double) * b->nprim, cudaMemcpyHostToDevice, st));
  HF_CUDA(cudaMemcpyAsync(dax.ptr, at_xyz.data(), sizeof(double) * 3 * b->natom, cudaMemcpyHostToDevice, st));
  const long long tot = (long long)n * n;
  one_electron_kernel<<<(unsigned)((tot + 127) / 128), 128, 0, st>>>(
      n, dbs.ptr, dl.ptr, dbf.ptr, dn.ptr, dp.ptr, dsx.ptr, dex.ptr, dco.ptr, b->natom, dax.ptr, dZ.ptr, ctx->boys64,
      ctx->rys, b->S.ptr, b->T.ptr, b->V.ptr);
  HF_CUDA(cudaGetLastError());
  HF_CUDA(cudaStreamSynchronize(st));
  b->have_one = true;
  return HF_OK;
}

extern "C" int hf_one_electron(hf_basis* b, double* S, double* T, double* V, double* e_nuc) {
  if (!b) return hf_fail(HF_ERR_INVALID, "null basis");
  hf_ctx* ctx = b->ctx;
  std::lock_guard<std::mutex> lk(ctx->mu);
  cudaSetDevice(ctx->device);
  HF_CHECK(hf_basis_one_electron(b));
  const size_t nn = (size_t)b->nbf * b->nbf * sizeof(double);
  if (S) HF_CUDA(cudaMemcpyAsync(S, b->S.ptr, nn, cudaMemcpyDeviceToDevice, ctx->stream));
  if (T) HF_CUDA(cudaMemcpyAsync(T, b->T.ptr, nn, cudaMemcpyDeviceToDevice, ctx->stream));
  if (V) HF_CUDA(cudaMemcpyAsync(V, b->V.ptr, nn, cudaMemcpyDeviceToDevice, ctx->stream));
  HF_CUDA(cudaStreamSynchronize(ctx->stream));
  if (e_nuc) *e_nuc = b->e_nuc;
  return HF_OK;
}
