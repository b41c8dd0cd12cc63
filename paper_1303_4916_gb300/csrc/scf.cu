// scf.cu -- closed-shell RHF iteration on the device.
//
// The procedure is Szabo-Ostlund's (the textbook the paper follows), with
// Pulay DIIS (Sec. "Technical details"):
//   X = S^{-1/2} = U s^{-1/2} U^T (symmetric Loewdin; lambda_min(S) < 1e-10
//   is HF_ERR_LINDEP); F_0 = H (core guess) or F(D0);
//   per iteration k: F' = X F X (X symmetric), F' C' = C' eps (cuSOLVER
//   syevd, ascending), C = X C', D = C_occ C_occ^T, J/K of D,
//   F_k = H + 2J - K, E_k = Tr[D (H + F_k)] + E_nuc; with DIIS the error
//   e_k = F_k D S - S D F_k and the most recent m (F, e) pairs give
//   F = sum c_i F_i from [B -1; -1 0][c; lambda] = [0; -1], B_ij = <e_i,e_j>
//   (oldest pair dropped while cond(B) > 1e14); stop at |E_k - E_{k-1}| <= e_tol.
//
// hf_scf_solve replays the J/K phase of each iteration from a CUDA graph.
// Matrices are symmetric except C and the DIIS products; cuBLAS works
// column-major, so a row-major symmetric buffer is read as itself.
#include <algorithm>
#include <cstdint>
#include <chrono>
#include <cstring>
#include <cmath>
#include <vector>

#include "hf_internal.h"
#include "multi.h"
#include "scf_internal.h"

namespace {

// F = H + jf J - K  (jf = 2 closed shell, 1 per spin of an unrestricted build)
__global__ void k_add_fock(const double* __restrict__ H, const double* __restrict__ J, const double* __restrict__ K,
                           double* __restrict__ F, size_t nn, double jf = 2.0) {
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t < nn) F[t] = H[t] + jf * J[t] - K[t];
}

__global__ void k_add(const double* __restrict__ A, const double* __restrict__ B, double* __restrict__ C, size_t nn) {
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t < nn) C[t] = A[t] + B[t];
}

// out[0] += sum D (H + F)   (out zeroed by the caller)
__global__ void k_energy(const double* __restrict__ D, const double* __restrict__ H, const double* __restrict__ F,
                         size_t nn, double* out) {
  double s = 0.0;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < nn; t += (size_t)gridDim.x * blockDim.x)
    s += D[t] * (H[t] + F[t]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ double ws[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) ws[w] = s;
  __syncthreads();
  if (w == 0) {
    s = lane < (int)(blockDim.x >> 5) ? ws[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) atomicAdd(out, s);
  }
}

// column k of the column-major U scaled by s_k^{-1/2}
__global__ void k_scale_cols(double* __restrict__ U, const double* __restrict__ s, int n) {
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= (size_t)n * n) return;
  const int k = (int)(t / n);
  U[t] *= 1.0 / sqrt(s[k]);
}

// e = M - M^T ; also max |e| into emax (as ordered bits of a non-negative double)
__global__ void k_antisym(const double* __restrict__ M, double* __restrict__ E, int n, unsigned long long* emax) {
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= (size_t)n * n) return;
  const int i = (int)(t / n), j = (int)(t % n);
  const double v = M[t] - M[(size_t)j * n + i];
  E[t] = v;
  atomicMax(emax, (unsigned long long)__double_as_longlong(fabs(v)));
}

// out[r] = <E_r, e> for r < m
__global__ void k_multi_dot(const double* __restrict__ ring, const int* __restrict__ slots, int m,
                            const double* __restrict__ e, size_t nn, double* out) {
  const int r = blockIdx.y;
  if (r >= m) return;
  const double* a = ring + (size_t)slots[r] * nn;
  double s = 0.0;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < nn; t += (size_t)gridDim.x * blockDim.x)
    s += a[t] * e[t];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ double ws[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) ws[w] = s;
  __syncthreads();
  if (w == 0) {
    s = lane < (int)(blockDim.x >> 5) ? ws[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) atomicAdd(out + r, s);
  }
}

__global__ void k_lincomb(const double* __restrict__ ring, const int* __restrict__ slots, const double* __restrict__ c,
                          int m, size_t nn, double* __restrict__ out) {
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= nn) return;
  double s = 0.0;
  for (int r = 0; r < m; ++r) s += c[r] * ring[(size_t)slots[r] * nn + t];
  out[t] = s;
}

// row-major copy of a column-major square matrix
__global__ void k_transpose(const double* __restrict__ A, double* __restrict__ B, int n) {
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= (size_t)n * n) return;
  const int i = (int)(t / n), j = (int)(t % n);
  B[t] = A[(size_t)j * n + i];
}

inline unsigned blocks(size_t n, int bs = 256) { return (unsigned)((n + bs - 1) / bs); }

// Eigenvalues of a small symmetric matrix (cyclic Jacobi), for cond(B).
void jacobi_eigs(std::vector<double> A, int n, std::vector<double>& w) {
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j) off += A[i * n + j] * A[i * n + j];
    if (off < 1e-300) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = A[p * n + q];
        if (apq == 0.0) continue;
        const double theta = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {
          const double akp = A[k * n + p], akq = A[k * n + q];
          A[k * n + p] = c * akp - s * akq;
          A[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {
          const double apk = A[p * n + k], aqk = A[q * n + k];
          A[p * n + k] = c * apk - s * aqk;
          A[q * n + k] = s * apk + c * aqk;
        }
      }
  }
  w.resize(n);
  for (int i = 0; i < n; ++i) w[i] = A[i * n + i];
}

// Solve A x = b (Gaussian elimination with partial pivoting). false if singular.
bool solve_small(std::vector<double> A, std::vector<double> b, int n, std::vector<double>& x) {
  for (int k = 0; k < n; ++k) {
    int piv = k;
    for (int i = k + 1; i < n; ++i)
      if (fabs(A[i * n + k]) > fabs(A[piv * n + k])) piv = i;
    if (A[piv * n + k] == 0.0) return false;
    if (piv != k) {
      for (int j = 0; j < n; ++j) std::swap(A[k * n + j], A[piv * n + j]);
      std::swap(b[k], b[piv]);
    }
    for (int i = k + 1; i < n; ++i) {
      const double f = A[i * n + k] / A[k * n + k];
      for (int j = k; j < n; ++j) A[i * n + j] -= f * A[k * n + j];
      b[i] -= f * b[k];
    }
  }
  x.assign(n, 0.0);
  for (int i = n - 1; i >= 0; --i) {
    double s = b[i];
    for (int j = i + 1; j < n; ++j) s -= A[i * n + j] * x[j];
    x[i] = s / A[i * n + i];
  }
  return true;
}

}  // namespace

// ------------------------------------------------------------- state
int scf_state_init(hf_basis* b, ScfState& s, int diis_size) {
  hf_ctx* ctx = b->ctx;
  const int n = b->nbf;
  const size_t nn = (size_t)n * n;
  s.n = n;
  s.m = std::max(0, std::min(diis_size, 16));
  HF_CHECK(s.H.alloc(ctx, nn));
  HF_CHECK(s.X.alloc(ctx, nn));
  HF_CHECK(s.F.alloc(ctx, nn));
  HF_CHECK(s.Fk.alloc(ctx, nn));
  HF_CHECK(s.W.alloc(ctx, nn));
  HF_CHECK(s.C.alloc(ctx, nn));
  HF_CHECK(s.D.alloc(ctx, nn));
  HF_CHECK(s.J.alloc(ctx, nn));
  HF_CHECK(s.K.alloc(ctx, nn));
  HF_CHECK(s.T1.alloc(ctx, nn));
  HF_CHECK(s.T2.alloc(ctx, nn));
  HF_CHECK(s.eps.alloc(ctx, n));
  HF_CHECK(s.scal.alloc(ctx, 40));
  HF_CHECK(s.islots.alloc(ctx, 16));
  HF_CHECK(s.info.alloc(ctx, 1));
  if (!s.hscal) {
    void* hp = nullptr;
    if (cudaMallocHost(&hp, sizeof(double) * 64 + sizeof(int) * 16) != cudaSuccess)
      return hf_fail(HF_ERR_OOM, "cudaMallocHost");
    s.hscal = static_cast<double*>(hp);
    s.hcoef = s.hscal + 32;
    s.hslots = reinterpret_cast<int*>(s.hscal + 64);
  }
  if (s.m > 0) {
    HF_CHECK(s.Fring.alloc(ctx, nn * s.m));
    HF_CHECK(s.Ering.alloc(ctx, nn * s.m));
  }
  int lw = 0;
  if (cusolverDnDsyevd_bufferSize(ctx->cusolver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, s.W.ptr, n,
                                  s.eps.ptr, &lw) != CUSOLVER_STATUS_SUCCESS)
    return hf_fail(HF_ERR_CUDA, "syevd_bufferSize");
  HF_CHECK(s.work.alloc(ctx, (size_t)std::max(lw, 1)));
  s.lwork = lw;
  return HF_OK;
}

static int syevd(hf_ctx* ctx, ScfState& s, double* A, double* w) {
  if (cusolverDnDsyevd(ctx->cusolver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, s.n, A, s.n, w, s.work.ptr,
                       s.lwork, s.info.ptr) != CUSOLVER_STATUS_SUCCESS)
    return hf_fail(HF_ERR_CUDA, "cusolverDnDsyevd failed");
  return HF_OK;
}

static int gemm(hf_ctx* ctx, cublasOperation_t ta, cublasOperation_t tb, int m, int n, int k, const double* A, int lda,
                const double* B, int ldb, double* C, int ldc) {
  const double one = 1.0, zero = 0.0;
  if (cublasDgemm(ctx->cublas, ta, tb, m, n, k, &one, A, lda, B, ldb, &zero, C, ldc) != CUBLAS_STATUS_SUCCESS)
    return hf_fail(HF_ERR_CUDA, "cublasDgemm failed");
  return HF_OK;
}

// H = T + V and X = S^{-1/2}; fills s.smin.
int scf_setup(hf_basis* b, ScfState& s) {
  hf_ctx* ctx = b->ctx;
  cudaStream_t st = ctx->stream;
  const int n = s.n;
  const size_t nn = (size_t)n * n;
  HF_CHECK(hf_basis_one_electron(b));
  k_add<<<blocks(nn), 256, 0, st>>>(b->T.ptr, b->V.ptr, s.H.ptr, nn);
  HF_CUDA(cudaMemcpyAsync(s.W.ptr, b->S.ptr, nn * sizeof(double), cudaMemcpyDeviceToDevice, st));
  HF_CHECK(syevd(ctx, s, s.W.ptr, s.eps.ptr));
  double smin = 0.0;
  HF_CUDA(cudaMemcpyAsync(&smin, s.eps.ptr, sizeof(double), cudaMemcpyDeviceToHost, st));
  HF_CUDA(cudaStreamSynchronize(st));
  s.smin = smin;
  if (!(smin >= 1e-10)) return hf_fail(HF_ERR_LINDEP, "lambda_min(S) = %.3e below 1e-10", smin);
  // X = (U s^{-1/2}) U^T
  HF_CUDA(cudaMemcpyAsync(s.T1.ptr, s.W.ptr, nn * sizeof(double), cudaMemcpyDeviceToDevice, st));
  k_scale_cols<<<blocks(nn), 256, 0, st>>>(s.T1.ptr, s.eps.ptr, n);
  HF_CHECK(gemm(ctx, CUBLAS_OP_N, CUBLAS_OP_T, n, n, n, s.T1.ptr, n, s.W.ptr, n, s.X.ptr, n));
  return HF_OK;
}

// Phase 1 of an iteration (enqueue only): from the current s.F,
// F' = X F X, eigen-decomposition, C = X C', D = C_occ C_occ^T.
int scf_density(hf_basis* b, ScfState& s) {
  hf_ctx* ctx = b->ctx;
  cudaStream_t st = ctx->stream;
  const int n = s.n, nocc = b->nelec / 2;
  const size_t nn = (size_t)n * n;
  HF_CHECK(gemm(ctx, CUBLAS_OP_N, CUBLAS_OP_N, n, n, n, s.F.ptr, n, s.X.ptr, n, s.T1.ptr, n));
  HF_CHECK(gemm(ctx, CUBLAS_OP_N, CUBLAS_OP_N, n, n, n, s.X.ptr, n, s.T1.ptr, n, s.W.ptr, n));
  HF_CHECK(syevd(ctx, s, s.W.ptr, s.eps.ptr));
  HF_CHECK(gemm(ctx, CUBLAS_OP_N, CUBLAS_OP_N, n, n, n, s.X.ptr, n, s.W.ptr, n, s.C.ptr, n));
  if (nocc > 0) {
    HF_CHECK(gemm(ctx, CUBLAS_OP_N, CUBLAS_OP_T, n, n, nocc, s.C.ptr, n, s.C.ptr, n, s.D.ptr, n));
  } else {
    HF_CUDA(cudaMemsetAsync(s.D.ptr, 0, nn * sizeof(double), st));
  }
  return HF_OK;
}

// Phase 2 (enqueue only, after J and K of D are in s.J, s.K):
// F_k = H + 2J - K, E_k, the DIIS error e_k = F D S - S D F, its dot
// products with the stored errors, and an asynchronous copy of these
// scalars to pinned host memory (s.hscal).
int scf_post_jk(hf_basis* b, ScfState& s) {
  hf_ctx* ctx = b->ctx;
  cudaStream_t st = ctx->stream;
  const int n = s.n;
  const size_t nn = (size_t)n * n;
  s.fock_builds += 1;
  k_add_fock<<<blocks(nn), 256, 0, st>>>(s.H.ptr, s.J.ptr, s.K.ptr, s.Fk.ptr, nn);
  HF_CUDA(cudaMemsetAsync(s.scal.ptr, 0, sizeof(double) * 40, st));
  k_energy<<<std::min(blocks(nn), 1024u), 256, 0, st>>>(s.D.ptr, s.H.ptr, s.Fk.ptr, nn, s.scal.ptr);
  HF_CHECK(gemm(ctx, CUBLAS_OP_N, CUBLAS_OP_N, n, n, n, s.D.ptr, n, b->S.ptr, n, s.T1.ptr, n));
  HF_CHECK(gemm(ctx, CUBLAS_OP_N, CUBLAS_OP_N, n, n, n, s.Fk.ptr, n, s.T1.ptr, n, s.T2.ptr, n));
  double* err = s.m > 0 ? s.Ering.ptr + (size_t)s.next * nn : s.T1.ptr;
  k_antisym<<<blocks(nn), 256, 0, st>>>(s.T2.ptr, err, n, (unsigned long long*)(s.scal.ptr + 1));
  if (s.m > 0) {
    HF_CUDA(cudaMemcpyAsync(s.Fring.ptr + (size_t)s.next * nn, s.Fk.ptr, nn * sizeof(double),
                            cudaMemcpyDeviceToDevice, st));
    s.slots.push_back(s.next);
    if ((int)s.slots.size() > s.m) s.slots.erase(s.slots.begin());
    s.next = (s.next + 1) % s.m;
    const int k = (int)s.slots.size();
    for (int i = 0; i < k; ++i) s.hslots[i] = s.slots[i];
    HF_CUDA(cudaMemcpyAsync(s.islots.ptr, s.hslots, sizeof(int) * k, cudaMemcpyHostToDevice, st));
    k_multi_dot<<<dim3(std::min(blocks(nn), 64u), k), 256, 0, st>>>(s.Ering.ptr, s.islots.ptr, k, err, nn,
                                                                    s.scal.ptr + 2);
  }
  HF_CUDA(cudaGetLastError());
  HF_CUDA(cudaMemcpyAsync(s.hscal, s.scal.ptr, sizeof(double) * 18, cudaMemcpyDeviceToHost, st));
  return HF_OK;
}

// DIIS on the host from the dot products in s.hscal, then enqueue the next
// F (extrapolated, or F_k) into Fout; vectors of len doubles (n^2, or 2 n^2
// for the stacked spins of an unrestricted SCF) in the rings.
static int diis_extrapolate(hf_basis* b, ScfState& s, size_t nn, double* Fout, const double* Fk) {
  hf_ctx* ctx = b->ctx;
  cudaStream_t st = ctx->stream;
  const double* sc = s.hscal;
  if (s.m > 0) {
    const int k = (int)s.slots.size();
    for (int i = 0; i < k; ++i)
      s.Bslot[s.slots[i] * 16 + s.slots[k - 1]] = s.Bslot[s.slots[k - 1] * 16 + s.slots[i]] = sc[2 + i];
    int first = 0;  // drop the oldest pairs while B is ill-conditioned
    std::vector<double> c;
    bool ok = false;
    while (k - first >= 2) {
      const int mm = k - first, na = mm + 1;
      std::vector<double> A(na * na, 0.0), rhs(na, 0.0), w;
      for (int i = 0; i < mm; ++i)
        for (int j = 0; j < mm; ++j) A[i * na + j] = s.Bslot[s.slots[first + i] * 16 + s.slots[first + j]];
      for (int i = 0; i < mm; ++i) A[i * na + mm] = A[mm * na + i] = -1.0;
      rhs[mm] = -1.0;
      jacobi_eigs(A, na, w);
      double amax = 0.0, amin = INFINITY;
      for (double x : w) {
        amax = std::max(amax, fabs(x));
        amin = std::min(amin, fabs(x));
      }
      if (amin == 0.0 || amax / amin > 1e14 || !solve_small(A, rhs, na, c)) {
        ++first;
        continue;
      }
      ok = true;
      break;
    }
    if (ok) {
      const int mm = k - first;
      for (int i = 0; i < mm; ++i) s.hcoef[i] = c[i];
      HF_CUDA(cudaMemcpyAsync(s.scal.ptr + 20, s.hcoef, sizeof(double) * mm, cudaMemcpyHostToDevice, st));
      k_lincomb<<<blocks(nn), 256, 0, st>>>(s.Fring.ptr, s.islots.ptr + first, s.scal.ptr + 20, mm, nn, Fout);
      HF_CUDA(cudaGetLastError());
      return HF_OK;
    }
  }
  HF_CUDA(cudaMemcpyAsync(Fout, Fk, nn * sizeof(double), cudaMemcpyDeviceToDevice, st));
  return HF_OK;
}

// Phase 3 (after the stream has passed phase 2): energy and DIIS
// bookkeeping on the host, then enqueue the next F (extrapolated or F_k).
int scf_diis_step(hf_basis* b, ScfState& s) {
  const double* sc = s.hscal;
  s.energy = sc[0] + b->e_nuc;
  s.diis_error = sc[1];  // bit pattern of a non-negative double: ordering preserved by atomicMax
  return diis_extrapolate(b, s, (size_t)s.n * s.n, s.F.ptr, s.Fk.ptr);
}

// One full iteration for a single molecule.
int scf_iterate(hf_basis* b, ScfState& s, const hf_scf_opts& o, const double* G) {
  HF_CHECK(scf_density(b, s));
  long long nq = 0;
  if (G) {
    HF_CHECK(hf_jk_stored_device(b, G, s.D.ptr, s.J.ptr, s.K.ptr));
  } else {
    HF_CHECK(hf_fock_jk_device(b, s.D.ptr, s.J.ptr, s.K.ptr, o.jk, &nq));
  }
  s.quartets += nq;
  HF_CHECK(scf_post_jk(b, s));
  HF_CUDA(cudaStreamSynchronize(b->ctx->stream));
  return scf_diis_step(b, s);
}

int scf_finish(hf_basis* b, ScfState& s, hf_scf_result* r) {
  hf_ctx* ctx = b->ctx;
  cudaStream_t st = ctx->stream;
  const int n = s.n, nocc = b->nelec / 2;
  const size_t nn = (size_t)n * n;
  r->energy = s.energy;
  r->e_nuc = b->e_nuc;
  r->e_elec = s.energy - b->e_nuc;
  r->delta_e = s.delta_e;
  r->diis_error = s.diis_error;
  r->iterations = s.iter;
  r->converged = s.converged;
  r->fock_builds = s.fock_builds;
  r->quartets = s.quartets;
  std::vector<double> eps(n);
  HF_CUDA(cudaMemcpyAsync(eps.data(), s.eps.ptr, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
  if (r->D) HF_CUDA(cudaMemcpyAsync(r->D, s.D.ptr, nn * sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (r->F) HF_CUDA(cudaMemcpyAsync(r->F, s.Fk.ptr, nn * sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (r->F1 && s.have_F1) HF_CUDA(cudaMemcpyAsync(r->F1, s.F1.ptr, nn * sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (r->eps) HF_CUDA(cudaMemcpyAsync(r->eps, s.eps.ptr, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  if (r->C) k_transpose<<<blocks(nn), 256, 0, st>>>(s.C.ptr, r->C, n);
  HF_CUDA(cudaStreamSynchronize(st));
  r->homo_lumo_gap = (nocc > 0 && nocc < n) ? eps[nocc] - eps[nocc - 1] : NAN;
  return HF_OK;
}

int scf_begin(hf_basis* b, ScfState& s, const hf_scf_opts& o, const double* G) {
  hf_ctx* ctx = b->ctx;
  cudaStream_t st = ctx->stream;
  const size_t nn = (size_t)s.n * s.n;
  HF_CHECK(scf_setup(b, s));
  s.iter = 0;
  s.converged = 0;
  s.energy = 0.0;
  s.e_old = NAN;
  s.delta_e = NAN;
  s.slots.clear();
  s.next = 0;
  s.fock_builds = 0;
  s.quartets = 0;
  s.have_F1 = false;
  if (o.D0) {
    HF_CUDA(cudaMemcpyAsync(s.D.ptr, o.D0, nn * sizeof(double), cudaMemcpyDeviceToDevice, st));
    long long nq = 0;
    if (G) HF_CHECK(hf_jk_stored_device(b, G, s.D.ptr, s.J.ptr, s.K.ptr));
    else HF_CHECK(hf_fock_jk_device(b, s.D.ptr, s.J.ptr, s.K.ptr, o.jk, &nq));
    s.quartets += nq;
    s.fock_builds += 1;
    k_add_fock<<<blocks(nn), 256, 0, st>>>(s.H.ptr, s.J.ptr, s.K.ptr, s.F.ptr, nn);
  } else {
    HF_CUDA(cudaMemcpyAsync(s.F.ptr, s.H.ptr, nn * sizeof(double), cudaMemcpyDeviceToDevice, st));
  }
  return HF_OK;
}

// After scf_iterate: bookkeeping of F_1, dE and convergence.  Returns true when done.
bool scf_after_iter(hf_basis* b, ScfState& s, const hf_scf_opts& o) {
  s.iter += 1;
  if (!s.have_F1) {
    const size_t nn = (size_t)s.n * s.n;
    if (s.F1.alloc(b->ctx, nn) == HF_OK &&
        cudaMemcpyAsync(s.F1.ptr, s.Fk.ptr, nn * sizeof(double), cudaMemcpyDeviceToDevice, b->ctx->stream) ==
            cudaSuccess)
      s.have_F1 = true;
  }
  if (!std::isnan(s.e_old)) {
    s.delta_e = fabs(s.energy - s.e_old);
    if (s.delta_e <= o.e_tol) {
      s.converged = 1;
      return true;
    }
  }
  s.e_old = s.energy;
  return s.iter >= o.max_iter;
}

extern "C" int hf_scf_solve(hf_basis* b, const hf_scf_opts* opts, hf_scf_result* res) {
  if (!b || !res) return hf_fail(HF_ERR_INVALID, "hf_scf_solve: null argument");
  if (b->nelec % 2)
    return hf_fail(HF_ERR_ODD_ELECTRONS, "closed-shell RHF needs an even electron count (%d)", b->nelec);
  hf_scf_opts o;
  hf_scf_opts_default(&o);
  if (opts) o = *opts;
  if (o.max_iter < 1 || o.diis_size < 0 || !(o.e_tol >= 0.0)) return hf_fail(HF_ERR_INVALID, "bad SCF options");
  HF_CHECK(hf_reject_deterministic(o.jk.flags, "hf_scf_solve"));
  hf_ctx* ctx = b->ctx;
  std::lock_guard<std::mutex> lk(ctx->mu);
  cudaSetDevice(ctx->device);
  const auto t0 = std::chrono::steady_clock::now();
  ScfState s;
  HF_CHECK(scf_state_init(b, s, o.diis_size));
  DevArray<double> G;
  if (o.flags & HF_SCF_STORED_ERI) {
    if (b->nbf > HF_STORED_NBF_MAX) return hf_fail(HF_ERR_INVALID, "stored ERI needs nbf <= %d", HF_STORED_NBF_MAX);
    HF_CHECK(G.alloc(ctx, (size_t)b->nbf * b->nbf * b->nbf * b->nbf));
    HF_CHECK(hf_eri_tensor_device(b, G.ptr));
  }
  HF_CHECK(scf_begin(b, s, o, G.ptr));
  // Direct J/K: the per-iteration J/K phase (zeroing, one launch per class,
  // symmetrisation) is captured once into a CUDA graph and replayed.
  MultiJK mj;
  const KernelCommon kc = hf_kernel_common(ctx, o.jk.flags);
  if (!G.ptr) {
    HF_CHECK(hf_basis_prepare_work(b, o.jk.schwarz_tau, o.jk.fp32_bound, o.jk.flags));
    mj.jk_flags = o.jk.flags;
    HF_CHECK(mj.build(ctx, {b}, {s.D.ptr}, {s.J.ptr}, {s.K.ptr}));
    HF_CHECK(mj.capture(kc));
  }
  for (;;) {
    NvtxRange nv("scf iteration (rhf)");
    if (G.ptr) {
      HF_CHECK(scf_iterate(b, s, o, G.ptr));
    } else {
      HF_CHECK(scf_density(b, s));
      HF_CHECK(mj.run(kc));
      s.quartets += mj.mol_quartets[0];
      HF_CHECK(scf_post_jk(b, s));
      HF_CUDA(cudaStreamSynchronize(ctx->stream));
      HF_CHECK(scf_diis_step(b, s));
    }
    const bool done = scf_after_iter(b, s, o);
    hf_log_scf_iter(ctx, "rhf", (unsigned long long)(uintptr_t)b, b->nbf, s.iter, s.energy, s.delta_e, s.diis_error,
                    std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(), s.converged);
    if (done) break;
  }
  HF_CHECK(scf_finish(b, s, res));
  res->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return s.converged ? HF_OK : hf_fail(HF_ERR_NOT_CONVERGED, "SCF not converged in %d iterations", s.iter);
}

// ------------------------------------------------------------- unrestricted HF
// Pople-Nesbet equations as Szabo-Ostlund state them (the paper's test
// calculations are UHF): per spin s with n_s electrons, D^s = C^s_occ
// C^s_occ^T, F^s = H + J[D^a + D^b] - K[D^s], E = (1/2) sum_s Tr[D^s (H +
// F^s)] + E_nuc; core guess F^a = F^b = H; with DIIS the two errors
// e^s = F^s D^s S - S D^s F^s are one stacked vector with one set of
// coefficients for both spins.  J, K^a and K^b come from one evaluation of
// the integrals per iteration (the J/K phase replayed from a CUDA graph).
// Buffers hold the two spins back to back: X2[0..n^2) alpha, [n^2..2n^2) beta.
namespace {

struct UhfState {
  ScfState s;  // shared: H, X, W, T1, T2, J, syevd workspace, scalars, DIIS rings (2 n^2 per slot)
  DevArray<double> F2, Fk2, C2, D2, K2, eps2, Dsum;
};

int uhf_init(hf_basis* b, UhfState& u, int diis_size) {
  hf_ctx* ctx = b->ctx;
  HF_CHECK(scf_state_init(b, u.s, 0));
  const size_t nn = (size_t)b->nbf * b->nbf;
  u.s.m = std::max(0, std::min(diis_size, 16));
  if (u.s.m > 0) {
    HF_CHECK(u.s.Fring.alloc(ctx, 2 * nn * u.s.m));
    HF_CHECK(u.s.Ering.alloc(ctx, 2 * nn * u.s.m));
  }
  HF_CHECK(u.F2.alloc(ctx, 2 * nn));
  HF_CHECK(u.Fk2.alloc(ctx, 2 * nn));
  HF_CHECK(u.C2.alloc(ctx, 2 * nn));
  HF_CHECK(u.D2.alloc(ctx, 2 * nn));
  HF_CHECK(u.K2.alloc(ctx, 2 * nn));
  HF_CHECK(u.eps2.alloc(ctx, 2 * (size_t)b->nbf));
  HF_CHECK(u.Dsum.alloc(ctx, nn));
  return HF_OK;
}

// F'^s = X F^s X, eigenvectors, C^s = X C'^s, D^s = C^s_occ C^s_occ^T, D^a + D^b.
int uhf_density(hf_basis* b, UhfState& u, const int nocc[2]) {
  hf_ctx* ctx = b->ctx;
  cudaStream_t st = ctx->stream;
  ScfState& s = u.s;
  const int n = s.n;
  const size_t nn = (size_t)n * n;
  for (int sp = 0; sp < 2; ++sp) {
    double* F = u.F2.ptr + sp * nn;
    double* Cm = u.C2.ptr + sp * nn;
    double* Dm = u.D2.ptr + sp * nn;
    HF_CHECK(gemm(ctx, CUBLAS_OP_N, CUBLAS_OP_N, n, n, n, F, n, s.X.ptr, n, s.T1.ptr, n));
    HF_CHECK(gemm(ctx, CUBLAS_OP_N, CUBLAS_OP_N, n, n, n, s.X.ptr, n, s.T1.ptr, n, s.W.ptr, n));
    HF_CHECK(syevd(ctx, s, s.W.ptr, u.eps2.ptr + (size_t)sp * n));
    HF_CHECK(gemm(ctx, CUBLAS_OP_N, CUBLAS_OP_N, n, n, n, s.X.ptr, n, s.W.ptr, n, Cm, n));
    if (nocc[sp] > 0) HF_CHECK(gemm(ctx, CUBLAS_OP_N, CUBLAS_OP_T, n, n, nocc[sp], Cm, n, Cm, n, Dm, n));
    else HF_CUDA(cudaMemsetAsync(Dm, 0, nn * sizeof(double), st));
  }
  k_add<<<blocks(nn), 256, 0, st>>>(u.D2.ptr, u.D2.ptr + nn, u.Dsum.ptr, nn);
  HF_CUDA(cudaGetLastError());
  return HF_OK;
}

// F^s = H + J - K^s, E (both spins into scal[0]), stacked DIIS error, dots.
int uhf_post_jk(hf_basis* b, UhfState& u) {
  hf_ctx* ctx = b->ctx;
  cudaStream_t st = ctx->stream;
  ScfState& s = u.s;
  const int n = s.n;
  const size_t nn = (size_t)n * n;
  s.fock_builds += 1;
  HF_CUDA(cudaMemsetAsync(s.scal.ptr, 0, sizeof(double) * 40, st));
  double* err = s.m > 0 ? s.Ering.ptr + (size_t)s.next * 2 * nn : nullptr;
  for (int sp = 0; sp < 2; ++sp) {
    double* Fk = u.Fk2.ptr + sp * nn;
    const double* Dm = u.D2.ptr + sp * nn;
    k_add_fock<<<blocks(nn), 256, 0, st>>>(s.H.ptr, s.J.ptr, u.K2.ptr + sp * nn, Fk, nn, 1.0);
    k_energy<<<std::min(blocks(nn), 1024u), 256, 0, st>>>(Dm, s.H.ptr, Fk, nn, s.scal.ptr);
    HF_CHECK(gemm(ctx, CUBLAS_OP_N, CUBLAS_OP_N, n, n, n, Dm, n, b->S.ptr, n, s.T1.ptr, n));
    HF_CHECK(gemm(ctx, CUBLAS_OP_N, CUBLAS_OP_N, n, n, n, Fk, n, s.T1.ptr, n, s.T2.ptr, n));
    k_antisym<<<blocks(nn), 256, 0, st>>>(s.T2.ptr, err ? err + sp * nn : s.T1.ptr, n,
                                          (unsigned long long*)(s.scal.ptr + 1));
  }
  if (s.m > 0) {
    HF_CUDA(cudaMemcpyAsync(s.Fring.ptr + (size_t)s.next * 2 * nn, u.Fk2.ptr, 2 * nn * sizeof(double),
                            cudaMemcpyDeviceToDevice, st));
    s.slots.push_back(s.next);
    if ((int)s.slots.size() > s.m) s.slots.erase(s.slots.begin());
    s.next = (s.next + 1) % s.m;
    const int k = (int)s.slots.size();
    for (int i = 0; i < k; ++i) s.hslots[i] = s.slots[i];
    HF_CUDA(cudaMemcpyAsync(s.islots.ptr, s.hslots, sizeof(int) * k, cudaMemcpyHostToDevice, st));
    k_multi_dot<<<dim3(std::min(blocks(2 * nn), 64u), k), 256, 0, st>>>(s.Ering.ptr, s.islots.ptr, k, err, 2 * nn,
                                                                        s.scal.ptr + 2);
  }
  HF_CUDA(cudaGetLastError());
  HF_CUDA(cudaMemcpyAsync(s.hscal, s.scal.ptr, sizeof(double) * 18, cudaMemcpyDeviceToHost, st));
  return HF_OK;
}

// <S^2> = S_z (S_z + 1) + n_b - sum_ij (C^a_occ^T S C^b_occ)_ij^2
int uhf_s2(hf_basis* b, UhfState& u, const int nocc[2], double* s2) {
  hf_ctx* ctx = b->ctx;
  ScfState& s = u.s;
  const int n = s.n;
  const size_t nn = (size_t)n * n;
  const double sz = 0.5 * (nocc[0] - nocc[1]);
  double ov2 = 0.0;
  if (nocc[0] > 0 && nocc[1] > 0) {
    HF_CHECK(gemm(ctx, CUBLAS_OP_N, CUBLAS_OP_N, n, nocc[1], n, b->S.ptr, n, u.C2.ptr + nn, n, s.T1.ptr, n));
    HF_CHECK(gemm(ctx, CUBLAS_OP_T, CUBLAS_OP_N, nocc[0], nocc[1], n, u.C2.ptr, n, s.T1.ptr, n, s.T2.ptr, nocc[0]));
    double nrm = 0.0;
    cublasPointerMode_t pm;
    cublasGetPointerMode(ctx->cublas, &pm);
    cublasSetPointerMode(ctx->cublas, CUBLAS_POINTER_MODE_HOST);
    const cublasStatus_t cs = cublasDnrm2(ctx->cublas, nocc[0] * nocc[1], s.T2.ptr, 1, &nrm);
    cublasSetPointerMode(ctx->cublas, pm);
    if (cs != CUBLAS_STATUS_SUCCESS) return hf_fail(HF_ERR_CUDA, "cublasDnrm2 failed");
    ov2 = nrm * nrm;
  }
  *s2 = sz * (sz + 1.0) + nocc[1] - ov2;
  return HF_OK;
}

}  // namespace

extern "C" int hf_uhf_solve(hf_basis* b, int n_alpha, int n_beta, const hf_scf_opts* opts, hf_uhf_result* res) {
  if (!b || !res) return hf_fail(HF_ERR_INVALID, "hf_uhf_solve: null argument");
  if (n_beta < 0 || n_alpha < n_beta || n_alpha > b->nbf)
    return hf_fail(HF_ERR_INVALID, "hf_uhf_solve: need nbf >= n_alpha >= n_beta >= 0 (%d, %d)", n_alpha, n_beta);
  hf_scf_opts o;
  hf_scf_opts_default(&o);
  if (opts) o = *opts;
  if (o.max_iter < 1 || o.diis_size < 0 || !(o.e_tol >= 0.0) || (o.flags & HF_SCF_STORED_ERI) || o.D0 ||
      (o.jk.flags & HF_JK_HOST))
    return hf_fail(HF_ERR_INVALID, "hf_uhf_solve: bad options (direct J/K, core guess, device buffers)");
  if (!(o.jk.schwarz_tau >= 0.0) || !(o.jk.fp32_bound >= 0.0)) return hf_fail(HF_ERR_INVALID, "negative threshold");
  HF_CHECK(hf_reject_deterministic(o.jk.flags, "hf_uhf_solve"));
  hf_ctx* ctx = b->ctx;
  std::lock_guard<std::mutex> lk(ctx->mu);
  cudaSetDevice(ctx->device);
  cudaStream_t st = ctx->stream;
  const auto t0 = std::chrono::steady_clock::now();
  const int nocc[2] = {n_alpha, n_beta};
  const size_t nn = (size_t)b->nbf * b->nbf;
  UhfState u;
  ScfState& s = u.s;
  HF_CHECK(uhf_init(b, u, o.diis_size));
  HF_CHECK(scf_setup(b, s));
  HF_CUDA(cudaMemcpyAsync(u.F2.ptr, s.H.ptr, nn * sizeof(double), cudaMemcpyDeviceToDevice, st));
  HF_CUDA(cudaMemcpyAsync(u.F2.ptr + nn, s.H.ptr, nn * sizeof(double), cudaMemcpyDeviceToDevice, st));
  HF_CHECK(hf_basis_prepare_work(b, o.jk.schwarz_tau, o.jk.fp32_bound, o.jk.flags));
  MultiJK mj;
  mj.jk_flags = o.jk.flags;
  const KernelCommon kc = hf_kernel_common(ctx, o.jk.flags);
  HF_CHECK(mj.build(ctx, {b}, {u.D2.ptr}, {s.J.ptr}, {u.K2.ptr}));
  HF_CHECK(mj.set_spin(0, u.Dsum.ptr, u.D2.ptr + nn, u.K2.ptr + nn));
  HF_CHECK(mj.capture(kc));
  s.iter = 0;
  s.e_old = NAN;
  s.delta_e = NAN;
  for (;;) {
    NvtxRange nv("scf iteration (uhf)");
    HF_CHECK(uhf_density(b, u, nocc));
    HF_CHECK(mj.run(kc));
    s.quartets += mj.mol_quartets[0];
    HF_CHECK(uhf_post_jk(b, u));
    HF_CUDA(cudaStreamSynchronize(st));
    s.energy = 0.5 * s.hscal[0] + b->e_nuc;
    s.diis_error = s.hscal[1];
    HF_CHECK(diis_extrapolate(b, s, 2 * nn, u.F2.ptr, u.Fk2.ptr));
    s.iter += 1;
    bool done = false;
    if (!std::isnan(s.e_old)) {
      s.delta_e = fabs(s.energy - s.e_old);
      if (s.delta_e <= o.e_tol) {
        s.converged = 1;
        done = true;
      }
    }
    s.e_old = s.energy;
    hf_log_scf_iter(ctx, "uhf", (unsigned long long)(uintptr_t)b, b->nbf, s.iter, s.energy, s.delta_e, s.diis_error,
                    std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(), s.converged);
    if (done || s.iter >= o.max_iter) break;
  }
  double s2 = 0.0;
  HF_CHECK(uhf_s2(b, u, nocc, &s2));
  res->energy = s.energy;
  res->e_nuc = b->e_nuc;
  res->e_elec = s.energy - b->e_nuc;
  res->delta_e = s.delta_e;
  res->diis_error = s.diis_error;
  res->s2 = s2;
  res->iterations = s.iter;
  res->converged = s.converged;
  res->fock_builds = s.fock_builds;
  res->quartets = s.quartets;
  if (res->Da) HF_CUDA(cudaMemcpyAsync(res->Da, u.D2.ptr, nn * sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (res->Db) HF_CUDA(cudaMemcpyAsync(res->Db, u.D2.ptr + nn, nn * sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (res->eps_a) HF_CUDA(cudaMemcpyAsync(res->eps_a, u.eps2.ptr, sizeof(double) * b->nbf, cudaMemcpyDeviceToDevice, st));
  if (res->eps_b)
    HF_CUDA(cudaMemcpyAsync(res->eps_b, u.eps2.ptr + b->nbf, sizeof(double) * b->nbf, cudaMemcpyDeviceToDevice, st));
  HF_CUDA(cudaStreamSynchronize(st));
  res->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return s.converged ? HF_OK : hf_fail(HF_ERR_NOT_CONVERGED, "UHF not converged in %d iterations", s.iter);
}
