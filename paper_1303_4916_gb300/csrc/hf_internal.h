// hf_internal.h -- host-side structures of libhf (not part of the ABI).
#pragma once
#include <cublas_v2.h>
#include <cuda_runtime.h>
#include <cusolverDn.h>

#include <nvtx3/nvToolsExt.h>

#include <atomic>
#include <cstdio>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/hf.h"
#include "hf_device.h"

// ------------------------------------------------------------- errors
int hf_fail(int code, const char* fmt, ...);  // records the message, returns code
#define HF_CUDA(call)                                                                              \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess) return hf_fail(HF_ERR_CUDA, "%s:%d %s: %s", __FILE__, __LINE__, #call, \
                                          cudaGetErrorString(e_));                                 \
  } while (0)
#define HF_CHECK(expr)         \
  do {                         \
    int rc_ = (expr);          \
    if (rc_ != HF_OK) return rc_; \
  } while (0)

// ------------------------------------------------------------- context
struct hf_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cublasHandle_t cublas = nullptr;
  cusolverDnHandle_t cusolver = nullptr;
  size_t hbm_budget = 0;
  int num_sms = 0;
  double* boys64 = nullptr;
  float* boys32 = nullptr;
  float* boysdf = nullptr;
  double* rys = nullptr;    // Rys roots and weights table (rys.cuh)
  EriClassOps ops[HF_NCLASS] = {};
  static constexpr int kSide = 4;
  cudaStream_t side[kSide] = {};     // class launches fork onto these (multi-molecule J/K)
  cudaEvent_t fork_ev = nullptr, join_ev[kSide] = {};
  std::atomic<int> fail_countdown{0};
  std::atomic<long long> device_bytes{0};
  std::mutex mu;  // serialises use of the stream-bound library handles
  int* bounds = nullptr;  // device status words of the bounds-checked build (2 ints)
  // bases and servers created on this context and not yet destroyed;
  // hf_ctx_destroy with live ones only marks the context, and the last
  // hf_basis_destroy / hf_serve_destroy tears it down (they free their
  // device memory through the context)
  std::atomic<int> live_bases{0};
  std::atomic<bool> destroy_pending{false};
  // JSON-lines log of SCF iterations (hf_ctx_set_log); null = off
  FILE* log = nullptr;
  bool own_log = false;
  std::mutex log_mu;
};

// NVTX range for the lifetime of a scope (a no-op unless a profiler is
// attached): J/K builds, class launches, SCF iterations.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Bounds-checked builds: the first failed index check since the last call
// (HF_ERR_INVALID with its code and index), else HF_OK; clears the status.
// Always HF_OK in the normal build.
int hf_bounds_status(hf_ctx* ctx, const char* where);

// One JSON line per SCF iteration into the context's log (when set):
// solver ("rhf", "uhf", "batch", "serve"), molecule tag, nbf, iteration,
// energy, |dE| (null on the first iteration), max DIIS error, seconds since
// the solve started, converged flag.
void hf_log_scf_iter(hf_ctx* ctx, const char* solver, unsigned long long mol, int nbf, int iter, double energy,
                     double delta_e, double diis_error, double t, int converged);
// One ready-made JSON object (no newline) into the context's log, when set.
void hf_log_line(hf_ctx* ctx, const char* json);

// Stream-ordered device allocation through the context (honours the
// fault-injection hook).  Returns HF_OK / HF_ERR_OOM.
int hf_dev_alloc(hf_ctx* ctx, void** p, size_t bytes);
// The teardown of hf_ctx_destroy (called when no basis is left).
void hf_ctx_teardown(hf_ctx* ctx);
void hf_dev_free(hf_ctx* ctx, void* p, size_t bytes);

template <typename T>
struct DevArray {
  T* ptr = nullptr;
  size_t n = 0;
  hf_ctx* ctx = nullptr;
  int alloc(hf_ctx* c, size_t count) {
    release();
    ctx = c;
    n = count;
    if (count == 0) return HF_OK;
    void* p = nullptr;
    int rc = hf_dev_alloc(c, &p, count * sizeof(T));
    if (rc != HF_OK) { n = 0; return rc; }
    ptr = static_cast<T*>(p);
    return HF_OK;
  }
  void release() {
    if (ptr) hf_dev_free(ctx, ptr, n * sizeof(T));
    ptr = nullptr;
    n = 0;
  }
  size_t bytes() const { return n * sizeof(T); }
  ~DevArray() { release(); }
};

// ------------------------------------------------------------- basis
struct ClassWork {
  DevArray<int> bra, kbeg, kend, ioff, nsplit;
  std::vector<int> bra_h, kbeg_h, kend_h, nsplit_h;  // host copies (multi-molecule launches, statistics)
  JKWork w{};
  long long nquartets = 0;
};

struct hf_basis {
  hf_ctx* ctx = nullptr;
  int natom = 0, nshell = 0, nbf = 0, nprim = 0, nelec = 0, lmax = 0;
  std::vector<hf_atom> atoms;
  std::vector<int> sh_atom, sh_l, sh_nprim, sh_prim, sh_bf;
  std::vector<double> exps, coefs;   // coefs: normalised, axial component
  double e_nuc = 0.0;

  // shell pairs, grouped by pair class, l_A >= l_B
  int npairs = 0, nprimpairs = 0;
  std::vector<int> pair_A, pair_B;
  int class_begin[HF_NPAIRCLASS + 1] = {};
  DevArray<double> prim64;
  DevArray<float> prim32;
  DevArray<float> primdf;
  DevArray<PairInfo> pinfo;
  DevArray<double> Q;                 // per pair
  std::vector<double> Q_h;
  std::vector<int> nprim_sig_h;
  DevArray<int> ketlist;              // per pair class: pair ids, primitive-count buckets, Q descending
  std::vector<int> ketlist_h;
  std::vector<int> buckets[HF_NPAIRCLASS];  // bucket boundaries (positions in the class list)

  // work lists for (tau, fp32_bound)
  bool have_work = false;
  double work_tau = -1.0, work_fp32 = -1.0;
  bool work_rys = false;
  ClassWork work64[HF_NCLASS], work32[HF_NCLASS];
  DevArray<int> counters;             // 2 * HF_NCLASS

  // scratch used by host-pointer J/K calls
  DevArray<double> hD, hJ, hK;
  // D^a + D^b of an unrestricted J/K call
  DevArray<double> Dsum;
  // fixed-point J', K' (and K2') accumulators of HF_JK_DETERMINISTIC builds,
  // two 64-bit words per element
  DevArray<unsigned long long> detq;

  // one-electron data (lazily)
  DevArray<double> S, T, V;
  bool have_one = false;
};

// Work lists for (tau, fp32_bound); HF_JK_RYS in flags builds every class's
// lists for the Rys kernel (one ket per item, items split into output
// chunks and primitive ranges), as the f/g classes always are.
int hf_basis_prepare_work(hf_basis* b, double tau, double fp32_bound, unsigned flags);

inline PairSet hf_pairset(const hf_basis* b) {
  return PairSet{b->prim64.ptr, b->prim32.ptr, b->pinfo.ptr, b->primdf.ptr, b->npairs, b->nprimpairs};
}
// Boys function of the reduced-precision (FP32) quartets: FP32 with
// HF_JK_FP32_BOYS; else df64 in the df64 tier (the tier's stand-in for FP64);
// else FP64.
inline KernelCommon hf_kernel_common(const hf_ctx* c, unsigned jk_flags) {
  const int f32 = (jk_flags & HF_JK_FP32_BOYS) ? 1 : 0;
  const int df = (!f32 && (jk_flags & HF_JK_DF64)) ? 1 : 0;
  return KernelCommon{c->boys64, c->boys32, f32, c->boysdf, df, 0, c->bounds, c->rys};  // det: set by hf_jk_run only
}
// HF_JK_DETERMINISTIC is served by hf_fock_jk, hf_fock_jk_profiled and
// hf_fock_jk_uhf; the entry points that build J/K elsewhere reject it.
inline int hf_reject_deterministic(unsigned jk_flags, const char* who) {
  return (jk_flags & HF_JK_DETERMINISTIC)
             ? hf_fail(HF_ERR_INVALID, "%s: HF_JK_DETERMINISTIC is served by hf_fock_jk and hf_fock_jk_uhf only", who)
             : HF_OK;
}
// launcher for the higher-precision work of a class: df64 when requested,
// the Rys route for every class under HF_JK_RYS
inline jk_launch_fn hf_jk_hi(const EriClassOps& op, unsigned jk_flags) {
  return (jk_flags & HF_JK_RYS) ? op.jkrys : (jk_flags & HF_JK_DF64) ? op.jkdf : op.jk64;
}
inline int hf_occ_hi(const EriClassOps& op, unsigned jk_flags) {
  return (jk_flags & HF_JK_RYS) ? op.occrys() : (jk_flags & HF_JK_DF64) ? op.occdf() : op.occ64();
}
// launcher for the reduced-precision (below fp32_bound) work of a class
inline jk_launch_fn hf_jk_lo(const EriClassOps& op, unsigned jk_flags) {
  return (jk_flags & HF_JK_RYS) ? op.jkrys : op.jk32;
}
inline int hf_occ_lo(const EriClassOps& op, unsigned jk_flags) {
  return (jk_flags & HF_JK_RYS) ? op.occrys() : op.occ32();
}
int hf_basis_one_electron(hf_basis* b);  // fills b->S, T, V
int hf_fock_jk_device(hf_basis* b, const double* D, double* J, double* K, const hf_jk_opts& o,
                      long long* nquartets);
// Grid of a persistent class launch: enough blocks of 4 warps for the work
// items, at most occ resident blocks on every SM.
int hf_launch_grid(hf_ctx* ctx, int occ, int nitems);
// Shape of a class launch of nitems work items: persistent 4-warp blocks
// that pull items from the counter, enough for the items and at most occ
// (or cap_per_sm when cap_per_sm > 0) resident blocks on every SM.  (One-warp
// blocks for classes with few items were measured on GB300 and did not
// shorten them: a small class is bound by its longest item.)
struct LaunchShape {
  int grid, threads;
};
LaunchShape hf_launch_shape(const hf_ctx* ctx, int occ, int nitems, int cap_per_sm = 0);
// CUDA events around each class launch of one J/K build (hf_fock_jk_profiled).
struct JKClassTiming {
  cudaEvent_t ev[2 * HF_NCLASS + 1];
  int which[2 * HF_NCLASS];
  int n = 0;
};
// The class kernels of one J/K build of b on stream st, for work lists
// already prepared for o: accumulates into Jp, Kp (zeroed by the caller)
// with the work-item counters at counters[0 .. 2*HF_NCLASS) (zeroed by the
// caller), then writes J = 2 (Jp + Jp^T), K = Kp + Kp^T (J == Jp and K == Kp
// for in place).  df64 and FP32 tiers as o.flags says.
// Second spin of an unrestricted build: J from Dj (D^a + D^b), and K2
// (zeroed by the caller, symmetrised in place) from D2.
struct JKSpin {
  const double* Dj;
  const double* D2;
  double* K2;
};
int hf_jk_run(hf_basis* b, const double* D, double* Jp, double* Kp, double* J, double* K, int* counters,
              const hf_jk_opts& o, cudaStream_t st, long long* nquartets, JKClassTiming* timing,
              const JKSpin* spin = nullptr);
int hf_boys_tables(hf_ctx* ctx);
int hf_eri_tensor_device(hf_basis* b, double* G);
int hf_jk_stored_device(hf_basis* b, const double* G, const double* D, double* J, double* K);
