// grad.cu -- analytic nuclear gradient of the closed-shell RHF energy (the
// paper's Hartree-Fock interatomic forces, which drive its structural
// relaxation and molecular dynamics; the force on an atom is -dE/dR).
//
// With D = C_occ C_occ^T (so E = Tr[D (H + F)] + E_nuc, F = H + 2J - K) and
// the energy-weighted density W = C_occ diag(eps_occ) C_occ^T, the gradient
// of the converged energy is
//   dE/dR = 2 sum_ij D_ij dH_ij/dR - 2 sum_ij W_ij dS_ij/dR
//         + sum over unique quartets Gamma d(ab|cd)/dR + dE_nuc/dR,
// the W term coming from the orthonormality of the orbitals.  The two-
// electron part runs on the Rys derivative kernel of every class
// (rys.cu); the one-electron part here, one thread per ordered pair (i, j)
// of basis functions, takes the derivatives with respect to the centre A
// of function i:
//   d phi_a / dA_x = 2 alpha phi_(a + 1_x) - a_x phi_(a - 1_x)
// applied to the Obara-Saika overlap and kinetic factors and to the
// Rys-quadrature nuclear attraction (a (i|1/r_C|j) with n = (la+lb+1)/2 + 1
// roots).  D, W, H and S are symmetric, so over all ordered pairs the
// derivatives with respect to the ket centre add up to those with respect
// to the bra centre: each thread adds twice its bra-centre term,
//   4 D_ij dH_ij/dA - 4 W_ij dS_ij/dA  to the atom of i,
// and the operator's own centre C (the Hellmann-Feynman term), whose
// derivative of (i|1/r_C|j) is -(d/dA + d/dB) by translational invariance,
// takes -4 D_ij d(i|1/r_C|j)/dA.
#include <cmath>
#include <vector>

#include "hf_internal.h"
#include "rys.cuh"

namespace {

__device__ __forceinline__ void cart_pow_g(int l, int c, int* p) {
  int k = 0;
  for (int x = l; x >= 0; --x)
    for (int y = l - x; y >= 0; --y) {
      if (k == c) { p[0] = x; p[1] = y; p[2] = l - x - y; return; }
      ++k;
    }
}

__device__ double comp_scale_g(int l, int c) {
  int p[3];
  cart_pow_g(l, c, p);
  auto df = [](int x) {
    double r = 1.0;
    for (int k = 2 * x - 1; k > 1; k -= 2) r *= k;
    return r;
  };
  return sqrt(df(l) / (df(p[0]) * df(p[1]) * df(p[2])));
}

__device__ double binom_g(int n, int k) {
  double r = 1.0;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return r;
}

// thread per ordered pair (i, j): one-electron gradient terms of the
// derivative with respect to the centre of i
__global__ void onee_grad_kernel(int nbf, const int* __restrict__ bf_shell, const int* __restrict__ sh_l,
                                 const int* __restrict__ sh_bf, const int* __restrict__ sh_nprim,
                                 const int* __restrict__ sh_prim, const int* __restrict__ sh_atom,
                                 const double* __restrict__ sh_xyz, const double* __restrict__ exps,
                                 const double* __restrict__ coefs, int natom, const double* __restrict__ atom_xyz,
                                 const int* __restrict__ atom_Z, const double* __restrict__ rys,
                                 const double* __restrict__ D, const double* __restrict__ W,
                                 double* __restrict__ grad) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)nbf * nbf) return;
  const int i = (int)(t / nbf), j = (int)(t % nbf);
  const double Dij = D[t], Wij = W[t];
  if (Dij == 0.0 && Wij == 0.0) return;
  const int sa = bf_shell[i], sb = bf_shell[j];
  const int la = sh_l[sa], lb = sh_l[sb];
  int pa[3], pb[3];
  cart_pow_g(la, i - sh_bf[sa], pa);
  cart_pow_g(lb, j - sh_bf[sb], pb);
  const double* A = sh_xyz + 3 * sa;
  const double* B = sh_xyz + 3 * sb;
  const double scale = comp_scale_g(la, i - sh_bf[sa]) * comp_scale_g(lb, j - sh_bf[sb]);
  double AB[3], r2 = 0.0;
  for (int x = 0; x < 3; ++x) {
    AB[x] = A[x] - B[x];
    r2 += AB[x] * AB[x];
  }
  double gS[3] = {0, 0, 0}, gT[3] = {0, 0, 0}, gV[3] = {0, 0, 0};
  double gVC[3 * 8];  // per nucleus, in rounds of 8
  const int L = la + lb + 1;
  const int nr = L / 2 + 1;
  for (int c0 = 0; c0 < natom; c0 += 8) {
    const int cn = min(8, natom - c0);
    for (int k = 0; k < 3 * cn; ++k) gVC[k] = 0.0;
    for (int ka = 0; ka < sh_nprim[sa]; ++ka)
      for (int kb = 0; kb < sh_nprim[sb]; ++kb) {
        const double a = exps[sh_prim[sa] + ka], b = exps[sh_prim[sb] + kb];
        const double c = coefs[sh_prim[sa] + ka] * coefs[sh_prim[sb] + kb] * scale;
        const double p = a + b, o2p = 0.5 / p, mu = a * b / p;
        double P[3], PA[3], PB[3];
        for (int x = 0; x < 3; ++x) {
          P[x] = (a * A[x] + b * B[x]) / p;
          PA[x] = P[x] - A[x];
          PB[x] = P[x] - B[x];
        }
        if (c0 == 0) {
          // 1D overlaps S[x][i][j], i <= la + 1, j <= lb + 2
          double S1[3][6][7];
          for (int x = 0; x < 3; ++x) {
            double (*s)[7] = S1[x];
            s[0][0] = sqrt(3.14159265358979323846 / p) * exp(-mu * AB[x] * AB[x]);
            for (int ii = 0; ii < pa[x] + 1; ++ii)
              s[ii + 1][0] = PA[x] * s[ii][0] + (ii > 0 ? ii * o2p * s[ii - 1][0] : 0.0);
            for (int ii = 0; ii <= pa[x] + 1; ++ii)
              for (int jj = 0; jj < pb[x] + 2; ++jj)
                s[ii][jj + 1] = PB[x] * s[ii][jj] +
                                ((ii > 0 ? ii * s[ii - 1][jj] : 0.0) + (jj > 0 ? jj * s[ii][jj - 1] : 0.0)) * o2p;
          }
          // kinetic factor of the ket on row ii
          auto tk = [&](int x, int ii) {
            const int jj = pb[x];
            double v = -2.0 * b * (2 * jj + 1) * S1[x][ii][jj] + 4.0 * b * b * S1[x][ii][jj + 2];
            if (jj >= 2) v += jj * (jj - 1) * S1[x][ii][jj - 2];
            return -0.5 * v;
          };
          double s0[3], t0[3], sd[3], td[3];
          for (int x = 0; x < 3; ++x) {
            s0[x] = S1[x][pa[x]][pb[x]];
            t0[x] = tk(x, pa[x]);
            sd[x] = 2.0 * a * S1[x][pa[x] + 1][pb[x]] - (pa[x] > 0 ? pa[x] * S1[x][pa[x] - 1][pb[x]] : 0.0);
            td[x] = 2.0 * a * tk(x, pa[x] + 1) - (pa[x] > 0 ? pa[x] * tk(x, pa[x] - 1) : 0.0);
          }
          for (int x = 0; x < 3; ++x) {
            const int y = (x + 1) % 3, z = (x + 2) % 3;
            gS[x] += c * sd[x] * s0[y] * s0[z];
            gT[x] += c * (td[x] * s0[y] * s0[z] + sd[x] * (t0[y] * s0[z] + s0[y] * t0[z]));
          }
        }
        // nuclear attraction by Rys quadrature: per root, 1D factors
        // I(i, j) from I(i+1) = (PA - u PC) I(i) + i (1-u)/(2p) I(i-1) and
        // the transfer to B
        const double pre = 2.0 * 3.14159265358979323846 / p * exp(-mu * r2);
        for (int cc = 0; cc < cn; ++cc) {
          const int at = c0 + cc;
          if (atom_Z[at] == 0) continue;
          const double* Cc = atom_xyz + 3 * at;
          const double PC[3] = {P[0] - Cc[0], P[1] - Cc[1], P[2] - Cc[2]};
          const double Tn = p * (PC[0] * PC[0] + PC[1] * PC[1] + PC[2] * PC[2]);
          double dv[3] = {0, 0, 0};
          for (int r = 0; r < nr; ++r) {
            double u, w;
            rys_rule_root(rys, nr, r, Tn, &u, &w);
            double v0[3], vd[3];
            for (int x = 0; x < 3; ++x) {
              double g[11];
              g[0] = 1.0;
              const double c00 = PA[x] - u * PC[x], b10 = (1.0 - u) * o2p;
              const int top = pa[x] + 1 + pb[x];
              for (int k = 0; k < top; ++k) g[k + 1] = c00 * g[k] + (k > 0 ? k * b10 * g[k - 1] : 0.0);
              auto tr = [&](int ii) {  // I(ii, pb) by the transfer to B
                double v = 0.0;
                for (int k = 0; k <= pb[x]; ++k) v += binom_g(pb[x], k) * pow(AB[x], pb[x] - k) * g[ii + k];
                return v;
              };
              v0[x] = tr(pa[x]);
              vd[x] = 2.0 * a * tr(pa[x] + 1) - (pa[x] > 0 ? pa[x] * tr(pa[x] - 1) : 0.0);
            }
            dv[0] += w * vd[0] * v0[1] * v0[2];
            dv[1] += w * v0[0] * vd[1] * v0[2];
            dv[2] += w * v0[0] * v0[1] * vd[2];
          }
          const double f = -(double)atom_Z[at] * c * pre;
          for (int x = 0; x < 3; ++x) {
            gV[x] += f * dv[x];
            gVC[3 * cc + x] += f * dv[x];
          }
        }
      }
    // the operator's centre
    for (int cc = 0; cc < cn; ++cc)
      for (int x = 0; x < 3; ++x)
        if (gVC[3 * cc + x] != 0.0) atomicAdd(grad + 3 * (c0 + cc) + x, -4.0 * Dij * gVC[3 * cc + x]);
  }
  const int ai = sh_atom[sa];
  for (int x = 0; x < 3; ++x) atomicAdd(grad + 3 * ai + x, 4.0 * Dij * (gT[x] + gV[x]) - 4.0 * Wij * gS[x]);
}

// rows of M = (row-major C)^T scaled by eps: Me(i, mu) = eps_i M(i, mu)
__global__ void scale_occ_rows(const double* __restrict__ M, const double* __restrict__ eps, int n, int nocc,
                               double* __restrict__ Me) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)n * n) return;
  const int i = (int)(t % n);  // column-major view: row index i = MO
  Me[t] = i < nocc ? eps[i] * M[t] : 0.0;
}

}  // namespace

extern "C" int hf_rhf_gradient(hf_basis* b, const double* C, const double* eps, int n_occ, const hf_jk_opts* opts,
                               double* grad_out) {
  if (!b || !C || !eps || !grad_out) return hf_fail(HF_ERR_INVALID, "hf_rhf_gradient: null argument");
  const int n = b->nbf;
  if (n_occ < 1 || n_occ > n) return hf_fail(HF_ERR_INVALID, "hf_rhf_gradient: n_occ %d outside [1, nbf]", n_occ);
  hf_jk_opts o;
  hf_jk_opts_default(&o);
  if (opts) o = *opts;
  if (o.flags & (HF_JK_HOST | HF_JK_DETERMINISTIC))
    return hf_fail(HF_ERR_INVALID, "hf_rhf_gradient: HF_JK_HOST and HF_JK_DETERMINISTIC are not taken");
  hf_ctx* ctx = b->ctx;
  std::lock_guard<std::mutex> lk(ctx->mu);
  HF_CUDA(cudaSetDevice(ctx->device));
  NvtxRange nv("RHF gradient");
  cudaStream_t st = ctx->stream;
  const size_t nn = (size_t)n * n;
  const int na = b->natom, ns = b->nshell;
  DevArray<double> D, W, Me, g, sx, ex, co, ax;
  DevArray<int> bfa, bfs, dl, dbf, dn, dp, dsa, dZ;
  HF_CHECK(D.alloc(ctx, nn));
  HF_CHECK(W.alloc(ctx, nn));
  HF_CHECK(Me.alloc(ctx, nn));
  HF_CHECK(g.alloc(ctx, 3 * (size_t)na));
  // D = C_occ C_occ^T and W = C_occ diag(eps) C_occ^T; the row-major C is
  // the column-major M = C^T, so D = M_occ^T M_occ
  const double one = 1.0, zero = 0.0;
  if (cublasDgemm(ctx->cublas, CUBLAS_OP_T, CUBLAS_OP_N, n, n, n_occ, &one, C, n, C, n, &zero, D.ptr, n) !=
      CUBLAS_STATUS_SUCCESS)
    return hf_fail(HF_ERR_CUDA, "cublasDgemm (density)");
  scale_occ_rows<<<(unsigned)((nn + 255) / 256), 256, 0, st>>>(C, eps, n, n_occ, Me.ptr);
  HF_CUDA(cudaGetLastError());
  if (cublasDgemm(ctx->cublas, CUBLAS_OP_T, CUBLAS_OP_N, n, n, n_occ, &one, Me.ptr, n, C, n, &zero, W.ptr, n) !=
      CUBLAS_STATUS_SUCCESS)
    return hf_fail(HF_ERR_CUDA, "cublasDgemm (energy-weighted density)");
  HF_CUDA(cudaMemsetAsync(g.ptr, 0, 3 * (size_t)na * sizeof(double), st));
  // one-electron terms
  std::vector<int> bf_shell(n), bf_atom(n), Z(na);
  for (int s = 0; s < ns; ++s)
    for (int k = b->sh_bf[s]; k < b->sh_bf[s + 1]; ++k) {
      bf_shell[k] = s;
      bf_atom[k] = b->sh_atom[s];
    }
  std::vector<double> sh_xyz(3 * ns), at_xyz(3 * na);
  for (int s = 0; s < ns; ++s)
    for (int x = 0; x < 3; ++x) sh_xyz[3 * s + x] = b->atoms[b->sh_atom[s]].xyz[x];
  for (int a = 0; a < na; ++a) {
    Z[a] = b->atoms[a].Z;
    for (int x = 0; x < 3; ++x) at_xyz[3 * a + x] = b->atoms[a].xyz[x];
  }
  HF_CHECK(bfa.alloc(ctx, n));
  HF_CHECK(bfs.alloc(ctx, n));
  HF_CHECK(dl.alloc(ctx, ns));
  HF_CHECK(dbf.alloc(ctx, ns + 1));
  HF_CHECK(dn.alloc(ctx, ns));
  HF_CHECK(dp.alloc(ctx, ns));
  HF_CHECK(dsa.alloc(ctx, ns));
  HF_CHECK(dZ.alloc(ctx, na));
  HF_CHECK(sx.alloc(ctx, 3 * ns));
  HF_CHECK(ex.alloc(ctx, b->nprim));
  HF_CHECK(co.alloc(ctx, b->nprim));
  HF_CHECK(ax.alloc(ctx, 3 * na));
#define UP(dst, src, cnt) HF_CUDA(cudaMemcpyAsync(dst.ptr, src, sizeof(*dst.ptr) * (cnt), cudaMemcpyHostToDevice, st))
  UP(bfa, bf_atom.data(), n);
  UP(bfs, bf_shell.data(), n);
  UP(dl, b->sh_l.data(), ns);
  UP(dbf, b->sh_bf.data(), ns + 1);
  UP(dn, b->sh_nprim.data(), ns);
  UP(dp, b->sh_prim.data(), ns);
  UP(dsa, b->sh_atom.data(), ns);
  UP(dZ, Z.data(), na);
  UP(sx, sh_xyz.data(), 3 * ns);
  UP(ex, b->exps.data(), b->nprim);
  UP(co, b->coefs.data(), b->nprim);
  UP(ax, at_xyz.data(), 3 * na);
#undef UP
  onee_grad_kernel<<<(unsigned)((nn + 127) / 128), 128, 0, st>>>(n, bfs.ptr, dl.ptr, dbf.ptr, dn.ptr, dp.ptr, dsa.ptr,
                                                                 sx.ptr, ex.ptr, co.ptr, na, ax.ptr, dZ.ptr, ctx->rys,
                                                                 D.ptr, W.ptr, g.ptr);
  HF_CUDA(cudaGetLastError());
  // two-electron terms: every class on the Rys derivative kernel, over the
  // Schwarz-screened unique quartets (Rys-shaped work lists)
  HF_CHECK(hf_basis_prepare_work(b, o.schwarz_tau, 0.0, HF_JK_RYS));
  HF_CUDA(cudaMemsetAsync(b->counters.ptr, 0, sizeof(int) * 2 * HF_NCLASS, st));
  const PairSet ps = hf_pairset(b);
  const KernelCommon kc = hf_kernel_common(ctx, 0);
  for (int c = HF_NCLASS - 1; c >= 0; --c) {
    const ClassWork& cw = b->work64[c];
    if (cw.w.nitems <= 0) continue;
    JKWork w = cw.w;
    w.counter = b->counters.ptr + 2 * c;
    NvtxRange nv_cls(ctx->ops[c].name ? ctx->ops[c].name : "class");
    ctx->ops[c].grad(w, ps, kc, D.ptr, bfa.ptr, n, g.ptr, 4 * ctx->num_sms, st);
  }
  HF_CUDA(cudaGetLastError());
  std::vector<double> gh(3 * (size_t)na);
  HF_CUDA(cudaMemcpyAsync(gh.data(), g.ptr, gh.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  HF_CUDA(cudaStreamSynchronize(st));
  HF_CHECK(hf_bounds_status(ctx, "RHF gradient"));
  // nuclear repulsion: dE_nuc/dR_a = -sum_b Z_a Z_b (R_a - R_b) / |R_a - R_b|^3
  for (int a = 0; a < na; ++a)
    for (int c = 0; c < na; ++c) {
      if (c == a) continue;
      double d[3], r2 = 0.0;
      for (int x = 0; x < 3; ++x) {
        d[x] = b->atoms[a].xyz[x] - b->atoms[c].xyz[x];
        r2 += d[x] * d[x];
      }
      if (r2 == 0.0) continue;
      const double f = (double)b->atoms[a].Z * b->atoms[c].Z / (r2 * std::sqrt(r2));
      for (int x = 0; x < 3; ++x) gh[3 * a + x] -= f * d[x];
    }
  for (size_t k = 0; k < gh.size(); ++k) grad_out[k] = gh[k];
  return HF_OK;
}
