// mp2.cu -- second-order Moller-Plesset correlation energy of a closed-shell
// RHF solution (the paper's MP2 follows Szabo-Ostlund), from the AO tensor
// held in HBM (nbf <= HF_STORED_NBF_MAX).
//
//   E(2) = sum_{i,j occ} sum_{a,b virt} (ia|jb) [2 (ia|jb) - (ib|ja)]
//                                        / (e_i + e_j - e_a - e_b)
//
// (ia|jb) comes from the AO tensor (ij|kl) of Eq. 5 (hf_eri_tensor) by four
// one-index transformations.  Each is one GEMM that contracts the leading
// index and appends the new one at the end,
//   out[X][t] = sum_p in[p][X] M[p][t],
// so that (pq|rs) -> [q r s i] -> [r s i a] -> [s i a j] -> [i a j b] with
// M = C_occ, C_virt, C_occ, C_virt in turn (cuBLAS DGEMM: plain dense
// contractions of the stored tensor), followed by one reduction kernel.
#include <cmath>

#include "hf_internal.h"

namespace {

// E(2) partial sums: V = (ia|jb) as V[((i*nv + a)*no + j)*nv + b].
__global__ void mp2_energy_kernel(const double* __restrict__ V, const double* __restrict__ eps, int no, int nv,
                                  double* out) {
  const long long tot = (long long)no * nv * no * nv;
  double s = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(t % nv);
    long long r = t / nv;
    const int j = (int)(r % no);
    r /= no;
    const int a = (int)(r % nv);
    const int i = (int)(r / nv);
    const double v = V[t];
    const double vx = V[(((long long)i * nv + b) * no + j) * nv + a];  // (ib|ja)
    s += v * (2.0 * v - vx) / (eps[i] + eps[j] - eps[no + a] - eps[no + b]);
  }
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

// out[X][t] = sum_p in[p][X] M[p][t]: in (n x L), M (n x T, row stride ldm),
// out (L x T), all row-major.  Column-major, out^T (T x L) = M^T (T x n) in (n x L).
int transform(hf_ctx* ctx, const double* in, long long L, const double* M, int T, int ldm, int n, double* out) {
  const double one = 1.0, zero = 0.0;
  if (L > 0x7fffffffLL) return hf_fail(HF_ERR_TOO_LARGE, "MP2 transform: %lld columns", L);
  if (cublasDgemm(ctx->cublas, CUBLAS_OP_N, CUBLAS_OP_T, T, (int)L, n, &one, M, ldm, in, (int)L, &zero, out, T) !=
      CUBLAS_STATUS_SUCCESS)
    return hf_fail(HF_ERR_CUDA, "cublasDgemm (MP2 transform) failed");
  return HF_OK;
}

}  // namespace

extern "C" int hf_mp2_energy(hf_basis* b, const double* C, const double* eps, int n_occ, double* e2) {
  if (!b || !C || !eps || !e2) return hf_fail(HF_ERR_INVALID, "hf_mp2_energy: null argument");
  const int n = b->nbf;
  if (n > HF_STORED_NBF_MAX)
    return hf_fail(HF_ERR_INVALID, "hf_mp2_energy: nbf %d above %d (stored AO tensor)", n, HF_STORED_NBF_MAX);
  if (n_occ < 1 || n_occ >= n) return hf_fail(HF_ERR_INVALID, "hf_mp2_energy: n_occ %d outside [1, nbf)", n_occ);
  hf_ctx* ctx = b->ctx;
  std::lock_guard<std::mutex> lk(ctx->mu);
  cudaSetDevice(ctx->device);
  cudaStream_t st = ctx->stream;
  const int no = n_occ, nv = n - n_occ;
  const size_t n4 = (size_t)n * n * n * n;
  const size_t t1 = (size_t)n * n * n * no;  // the largest intermediate
  DevArray<double> G, A, Bf, out;
  HF_CHECK(G.alloc(ctx, n4));
  HF_CHECK(A.alloc(ctx, t1));
  HF_CHECK(Bf.alloc(ctx, std::max((size_t)n * n * no * nv, (size_t)1)));
  HF_CHECK(out.alloc(ctx, 1));
  HF_CHECK(hf_eri_tensor_device(b, G.ptr));
  const long long nn = (long long)n * n;
  // (pq|rs) -> T1[q r s i] -> T2[r s i a] -> T3[s i a j] -> V[i a j b]
  HF_CHECK(transform(ctx, G.ptr, nn * n, C, no, n, n, A.ptr));
  HF_CHECK(transform(ctx, A.ptr, nn * no, C + no, nv, n, n, Bf.ptr));
  HF_CHECK(transform(ctx, Bf.ptr, (long long)n * no * nv, C, no, n, n, A.ptr));
  HF_CHECK(transform(ctx, A.ptr, (long long)no * nv * no, C + no, nv, n, n, Bf.ptr));
  HF_CUDA(cudaMemsetAsync(out.ptr, 0, sizeof(double), st));
  mp2_energy_kernel<<<std::min(1024LL, ((long long)no * nv * no * nv + 255) / 256 + 1), 256, 0, st>>>(
      Bf.ptr, eps, no, nv, out.ptr);
  HF_CUDA(cudaGetLastError());
  HF_CUDA(cudaMemcpyAsync(e2, out.ptr, sizeof(double), cudaMemcpyDeviceToHost, st));
  HF_CUDA(cudaStreamSynchronize(st));
  return HF_OK;
}
