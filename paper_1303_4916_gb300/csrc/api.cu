// api.cu -- context, error reporting, device allocation, Boys tables.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "hf_internal.h"
#include "rys.cuh"

static thread_local std::string g_last_error;

int hf_fail(int code, const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

extern "C" const char* hf_last_error(void) { return g_last_error.c_str(); }

extern "C" const char* hf_strerror(int code) {
  switch (code) {
    case HF_OK: return "ok";
    case HF_PENDING: return "pending";
    case HF_ERR_INVALID: return "invalid argument";
    case HF_ERR_UNSUPPORTED_L: return "unsupported angular momentum";
    case HF_ERR_OOM: return "out of memory";
    case HF_ERR_LINDEP: return "linearly dependent basis";
    case HF_ERR_NOT_CONVERGED: return "SCF not converged";
    case HF_ERR_TIMEOUT: return "timeout";
    case HF_ERR_CUDA: return "CUDA error";
    case HF_ERR_ODD_ELECTRONS: return "odd electron count";
    case HF_ERR_NOT_FOUND: return "not found";
    case HF_ERR_QUEUE_FULL: return "queue full";
    case HF_ERR_CANCELLED: return "cancelled";
    case HF_ERR_TOO_LARGE: return "request exceeds the memory budget or a work-list limit";
    default: return "unknown error";
  }
}

extern "C" void hf_jk_opts_default(hf_jk_opts* o) {
  if (!o) return;
  o->schwarz_tau = 1e-12;
  o->fp32_bound = 0.0;
  o->flags = 0;
}

extern "C" void hf_scf_opts_default(hf_scf_opts* o) {
  if (!o) return;
  o->max_iter = 128;
  o->e_tol = 1e-8;
  o->diis_size = 8;
  o->D0 = nullptr;
  hf_jk_opts_default(&o->jk);
  o->flags = 0;
}

int hf_dev_alloc(hf_ctx* ctx, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) return HF_OK;
  int c = ctx->fail_countdown.load();
  if (c > 0) {
    if (ctx->fail_countdown.fetch_sub(1) == 1)
      return hf_fail(HF_ERR_OOM, "injected allocation failure (%zu bytes)", bytes);
  }
  cudaError_t e = cudaMallocAsync(p, bytes, ctx->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return hf_fail(HF_ERR_OOM, "cudaMallocAsync(%zu): %s", bytes, cudaGetErrorString(e));
  }
  ctx->device_bytes += (long long)bytes;
  return HF_OK;
}

void hf_dev_free(hf_ctx* ctx, void* p, size_t bytes) {
  if (!p) return;
  cudaFreeAsync(p, ctx->stream);
  ctx->device_bytes -= (long long)bytes;
}

// ------------------------------------------------------------- Boys table
// F_m(T), m = 0..BOYS_NM-1, and exp(-T) in long double: F_{NM-1}(T) from its
// power series
//   F_m(T) = exp(-T) sum_k (2T)^k / ((2m+1)(2m+3)...(2m+2k+1)),
// the lower orders by the downward recursion F_m = (2T F_{m+1} + e^{-T})/(2m+1),
// which is stable in that direction.
static void boys_row(long double T, long double* F, long double* et) {
  const int M = BOYS_NM - 1;
  long double term = 1.0L / (2 * M + 1), sum = term;
  for (int k = 1; k < 5000; ++k) {
    term *= 2.0L * T / (long double)(2 * M + 2 * k + 1);
    sum += term;
    if (term <= sum * 1e-21L) break;
  }
  *et = expl(-T);
  F[M] = *et * sum;
  for (int m = M - 1; m >= 0; --m) F[m] = (2.0L * T * F[m + 1] + *et) / (long double)(2 * m + 1);
}

int hf_boys_tables(hf_ctx* ctx) {
  const size_t n64 = (size_t)(BOYS_LMAX + 1) * BOYS_NGRID * BOYS64_ROW;
  const size_t n32 = (size_t)(BOYS_LMAX + 1) * BOYS_NGRID * BOYS32_ROW;
  std::vector<double> t64(n64);
  std::vector<float> t32(n32);
  long double F[BOYS_NM], et;
  long double fact[BOYS64_TERMS];
  fact[0] = 1.0L;
  for (int k = 1; k < BOYS64_TERMS; ++k) fact[k] = fact[k - 1] * k;
  for (int i = 0; i < BOYS_NGRID; ++i) {
    boys_row((long double)((double)i * BOYS_H), F, &et);
    for (int L = 0; L <= BOYS_LMAX; ++L) {
      double* r = &t64[((size_t)L * BOYS_NGRID + i) * BOYS64_ROW];
      for (int k = 0; k < BOYS64_TERMS; ++k) {
        r[k] = (double)(F[L + k] / fact[k]);
        r[BOYS64_TERMS + k] = (double)(et / fact[k]);
      }
      float* f = &t32[((size_t)L * BOYS_NGRID + i) * BOYS32_ROW];
      for (int k = 0; k < BOYS32_TERMS; ++k) {
        f[k] = (float)(F[L + k] / fact[k]);
        f[BOYS32_TERMS + k] = (float)(et / fact[k]);
      }
    }
  }
  // df64 table: grid T_i = i/16, per (order, row) 16 floats: the Taylor
  // coefficients of F_L (c_0..c_4 as hi/lo pairs, c_5..c_7 as floats), a pad,
  // and exp(-T_i) as a hi/lo pair
  const size_t ndf = (size_t)(BOYS_LMAX + 1) * BOYSDF_NGRID * BOYSDF_ROW;
  std::vector<float> tdf(ndf, 0.0f);
  auto split = [](long double c, float* q) {
    const float h = (float)c;
    q[0] = h;
    q[1] = (float)(c - (long double)h);
  };
  for (int i = 0; i < BOYSDF_NGRID; ++i) {
    boys_row((long double)i / 16.0L, F, &et);
    for (int L = 0; L <= BOYS_LMAX; ++L) {
      float* r = &tdf[((size_t)L * BOYSDF_NGRID + i) * BOYSDF_ROW];
      for (int k = 0; k < 8; ++k) {
        const long double c = F[L + k] / fact[k];
        if (k < 5) split(c, r + 2 * k);
        else r[10 + (k - 5)] = (float)c;
      }
      split(et, r + 14);
    }
  }
  void* p = nullptr;
  HF_CHECK(hf_dev_alloc(ctx, &p, ndf * sizeof(float)));
  ctx->boysdf = (float*)p;
  HF_CUDA(cudaMemcpyAsync(ctx->boysdf, tdf.data(), ndf * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
  HF_CHECK(hf_dev_alloc(ctx, &p, n64 * sizeof(double)));
  ctx->boys64 = (double*)p;
  HF_CHECK(hf_dev_alloc(ctx, &p, n32 * sizeof(float)));
  ctx->boys32 = (float*)p;
  HF_CUDA(cudaMemcpyAsync(ctx->boys64, t64.data(), n64 * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  HF_CUDA(cudaMemcpyAsync(ctx->boys32, t32.data(), n32 * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
  HF_CUDA(cudaStreamSynchronize(ctx->stream));
  return HF_OK;
}

// ------------------------------------------------------------- context
extern "C" int hf_ctx_create(hf_ctx** out, int device, size_t hbm_budget, void* cuda_stream) {
  if (!out) return hf_fail(HF_ERR_INVALID, "hf_ctx_create: out is NULL");
  *out = nullptr;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return hf_fail(HF_ERR_CUDA, "no CUDA device: %s", cudaGetErrorString(e));
  }
  if (device < 0 || device >= ndev) return hf_fail(HF_ERR_INVALID, "device %d out of range (%d)", device, ndev);
  hf_ctx* c = new (std::nothrow) hf_ctx();
  if (!c) return hf_fail(HF_ERR_OOM, "host allocation");
  c->device = device;
  int rc = HF_OK;
  do {
    if (cudaSetDevice(device) != cudaSuccess) { rc = hf_fail(HF_ERR_CUDA, "cudaSetDevice"); break; }
    if (cuda_stream) {
      c->stream = (cudaStream_t)cuda_stream;
    } else {
      // a blocking stream: ordered after work on the legacy default stream
      // (where a caller such as PyTorch may have written the inputs)
      if (cudaStreamCreate(&c->stream) != cudaSuccess) {
        rc = hf_fail(HF_ERR_CUDA, "cudaStreamCreate");
        break;
      }
      c->own_stream = true;
    }
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    c->hbm_budget = hbm_budget ? hbm_budget : (size_t)(0.8 * (double)fr);
    if (cublasCreate(&c->cublas) != CUBLAS_STATUS_SUCCESS) { rc = hf_fail(HF_ERR_CUDA, "cublasCreate"); break; }
    cublasSetStream(c->cublas, c->stream);
    if (cusolverDnCreate(&c->cusolver) != CUSOLVER_STATUS_SUCCESS) {
      rc = hf_fail(HF_ERR_CUDA, "cusolverDnCreate");
      break;
    }
    cusolverDnSetStream(c->cusolver, c->stream);
    for (int k = 0; k < hf_ctx::kSide && rc == HF_OK; ++k) {
      if (cudaStreamCreateWithFlags(&c->side[k], cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&c->join_ev[k], cudaEventDisableTiming) != cudaSuccess)
        rc = hf_fail(HF_ERR_CUDA, "side stream");
    }
    if (rc == HF_OK && cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming) != cudaSuccess)
      rc = hf_fail(HF_ERR_CUDA, "fork event");
    if (rc != HF_OK) break;
    hf_register_classes_sp(c->ops);
    hf_register_classes_d1(c->ops);
    hf_register_classes_d2(c->ops);
    hf_register_classes_d3(c->ops);
    hf_register_classes_d4(c->ops);
    hf_register_classes_d5(c->ops);
    hf_register_classes_d6(c->ops);
    hf_register_classes_rys(c->ops);
    for (int k = 0; k < HF_NCLASS; ++k)
      if (!c->ops[k].jk64) { rc = hf_fail(HF_ERR_CUDA, "class %d has no kernels", k); break; }
    if (rc != HF_OK) break;
    rc = hf_boys_tables(c);
    if (rc != HF_OK) break;
    {
      void* rp = nullptr;
      rc = hf_dev_alloc(c, &rp, RYS_TAB_DOUBLES * sizeof(double));
      if (rc != HF_OK) break;
      c->rys = static_cast<double*>(rp);
      if (cudaMemcpyAsync(c->rys, hf_rys_table_host(), RYS_TAB_DOUBLES * sizeof(double), cudaMemcpyHostToDevice,
                          c->stream) != cudaSuccess)
        rc = hf_fail(HF_ERR_CUDA, "Rys table upload");
      if (rc != HF_OK) break;
    }
    void* bp = nullptr;
    rc = hf_dev_alloc(c, &bp, 2 * sizeof(int));
    if (rc != HF_OK) break;
    c->bounds = static_cast<int*>(bp);
    if (cudaMemsetAsync(c->bounds, 0, 2 * sizeof(int), c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
      rc = hf_fail(HF_ERR_CUDA, "bounds status");
  } while (0);
  if (rc != HF_OK) {
    hf_ctx_destroy(c);
    return rc;
  }
  *out = c;
  return HF_OK;
}

extern "C" void hf_ctx_destroy(hf_ctx* c) {
  if (!c) return;
  // bases still alive free their memory through this context: the last of
  // them completes the teardown
  c->destroy_pending.store(true);
  if (c->live_bases.load() > 0) return;
  hf_ctx_teardown(c);
}

void hf_ctx_teardown(hf_ctx* c) {
  cudaSetDevice(c->device);
  if (c->boys64) hf_dev_free(c, c->boys64, 0);
  if (c->boys32) hf_dev_free(c, c->boys32, 0);
  if (c->boysdf) hf_dev_free(c, c->boysdf, 0);
  if (c->rys) hf_dev_free(c, c->rys, 0);
  if (c->bounds) hf_dev_free(c, c->bounds, 0);
  if (c->stream) cudaStreamSynchronize(c->stream);
  for (int k = 0; k < hf_ctx::kSide; ++k) {
    if (c->side[k]) cudaStreamDestroy(c->side[k]);
    if (c->join_ev[k]) cudaEventDestroy(c->join_ev[k]);
  }
  if (c->fork_ev) cudaEventDestroy(c->fork_ev);
  if (c->cublas) cublasDestroy(c->cublas);
  if (c->cusolver) cusolverDnDestroy(c->cusolver);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  if (c->log && c->own_log) fclose(c->log);
  delete c;
}

int hf_bounds_status(hf_ctx* c, const char* where) {
#ifdef HF_BOUNDS_CHECK
  int st[2] = {0, 0};
  HF_CUDA(cudaMemcpyAsync(st, c->bounds, sizeof st, cudaMemcpyDeviceToHost, c->stream));
  HF_CUDA(cudaStreamSynchronize(c->stream));
  if (st[0] != 0) {
    HF_CUDA(cudaMemsetAsync(c->bounds, 0, sizeof st, c->stream));
    static const char* names[] = {"", "work item", "shell pair", "primitive record", "matrix element", "Boys row"};
    return hf_fail(HF_ERR_INVALID, "%s: bounds check failed: %s index %d", where,
                   st[0] > 0 && st[0] < 6 ? names[st[0]] : "?", st[1]);
  }
#else
  (void)c;
  (void)where;
#endif
  return HF_OK;
}

extern "C" int hf_bounds_checked(void) {
#ifdef HF_BOUNDS_CHECK
  return 1;
#else
  return 0;
#endif
}

extern "C" int hf_ctx_set_log(hf_ctx* c, const char* path) {
  if (!c) return hf_fail(HF_ERR_INVALID, "hf_ctx_set_log: null context");
  std::lock_guard<std::mutex> lk(c->log_mu);
  if (c->log && c->own_log) fclose(c->log);
  c->log = nullptr;
  c->own_log = false;
  if (!path) return HF_OK;
  if (path[0] == '-' && path[1] == 0) {
    c->log = stderr;
    return HF_OK;
  }
  FILE* f = fopen(path, "a");
  if (!f) return hf_fail(HF_ERR_INVALID, "hf_ctx_set_log: cannot open %s", path);
  c->log = f;
  c->own_log = true;
  return HF_OK;
}

void hf_log_scf_iter(hf_ctx* c, const char* solver, unsigned long long mol, int nbf, int iter, double energy,
                     double delta_e, double diis_error, double t, int converged) {
  if (!c || !c->log) return;
  std::lock_guard<std::mutex> lk(c->log_mu);
  if (!c->log) return;
  char de[40];
  if (delta_e == delta_e) snprintf(de, sizeof de, "%.17g", delta_e);
  else snprintf(de, sizeof de, "null");
  fprintf(c->log,
          "{\"event\": \"scf_iter\", \"solver\": \"%s\", \"mol\": %llu, \"nbf\": %d, \"iter\": %d, "
          "\"energy\": %.17g, \"delta_e\": %s, \"diis_error\": %.6g, \"t\": %.6f, \"converged\": %d}\n",
          solver, mol, nbf, iter, energy, de, diis_error, t, converged);
  fflush(c->log);
}

void hf_log_line(hf_ctx* c, const char* json) {
  if (!c || !c->log) return;
  std::lock_guard<std::mutex> lk(c->log_mu);
  if (!c->log) return;
  fprintf(c->log, "%s\n", json);
  fflush(c->log);
}

extern "C" void* hf_ctx_stream(hf_ctx* c) { return c ? (void*)c->stream : nullptr; }
extern "C" int hf_ctx_num_sms(hf_ctx* c) { return c ? c->num_sms : 0; }
extern "C" void hf_ctx_inject_alloc_failure(hf_ctx* c, int n) {
  if (c) c->fail_countdown.store(n > 0 ? n : 0);
}
