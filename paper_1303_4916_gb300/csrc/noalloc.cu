// noalloc.cu -- a J/K build for callers that cannot allocate device memory.
//
// hf_fock_jk accumulates into the caller's J and K and keeps its work-item
// counters in memory the basis handle allocated.  Some callers cannot call
// cudaMalloc at the point where they need a Fock build: code running under
// an allocator that is frozen after start-up, a host framework that owns all
// device memory and hands out only its own buffers, or a real-time loop that
// must not hit the allocator.  hf_fock_jk_noalloc serves them: its scratch
// (the J' and K' accumulators and the work-item counters) lives in one
// file-scope static device array below, so the call allocates nothing.
//
// Limits and rules (also stated in include/hf.h):
//   - nbf <= HF_NOALLOC_MAX_NBF (512); larger bases get HF_ERR_TOO_LARGE.
//   - The static array (2 * 512^2 doubles + counters, about 4 MiB) is held by
//     every GPU that loads the library until the process exits.
//   - The first call on a device looks up the array's device address with
//     cudaGetSymbolAddress (once per device); make that first call before
//     any stream capture.
//   - Every call shares the one array: calls that overlap on the GPU (other
//     threads, other contexts on the same device) race.  Each call clears
//     the part it uses before the kernels run.
//   - The quartet work lists for the given options must already exist on
//     the basis (hf_fock_jk or hf_count_quartets with the same options
//     builds them); otherwise HF_ERR_INVALID, since building them allocates.
#include <mutex>

#include "hf_internal.h"

#define HF_NOALLOC_MAX_NBF 512
#define HF_NOALLOC_NN ((size_t)HF_NOALLOC_MAX_NBF * HF_NOALLOC_MAX_NBF)
#define HF_NOALLOC_COUNTER_DOUBLES 128  // room for 2 * HF_NCLASS int counters

// [0, NN): J' ; [NN, 2NN): K' ; then the work-item counters (as int).
static_assert(HF_NOALLOC_COUNTER_DOUBLES * 2 >= 2 * HF_NCLASS, "counter room");
static __device__ __align__(256) double g_noalloc_scratch[2 * HF_NOALLOC_NN + HF_NOALLOC_COUNTER_DOUBLES];

namespace {

std::mutex g_setup_mu;
double* g_scratch_addr[256] = {};

// Device address of the static array for the current device (looked up once
// per device and kept for the life of the process; a cudaDeviceReset of that
// device unloads the module and leaves the kept address stale, so the entry
// point must not be used after one).
int noalloc_scratch(int device, double** out) {
  if (device < 0 || device >= 256) return hf_fail(HF_ERR_INVALID, "device index %d", device);
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (!g_scratch_addr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return hf_fail(HF_ERR_CUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
    g_scratch_addr[device] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[device];
  return HF_OK;
}

}  // namespace

extern "C" int hf_fock_jk_noalloc(hf_basis* b, const double* D, double* J, double* K, const hf_jk_opts* opts) {
  if (!b || !D || !J || !K) return hf_fail(HF_ERR_INVALID, "hf_fock_jk_noalloc: null argument");
  hf_jk_opts o;
  hf_jk_opts_default(&o);
  if (opts) o = *opts;
  if (!(o.schwarz_tau >= 0.0) || !(o.fp32_bound >= 0.0)) return hf_fail(HF_ERR_INVALID, "negative threshold");
  if (o.flags & HF_JK_HOST)
    return hf_fail(HF_ERR_INVALID, "hf_fock_jk_noalloc: device pointers only (HF_JK_HOST needs staging buffers)");
  HF_CHECK(hf_reject_deterministic(o.flags, "hf_fock_jk_noalloc"));
  const int n = b->nbf;
  if (n > HF_NOALLOC_MAX_NBF)
    return hf_fail(HF_ERR_TOO_LARGE, "hf_fock_jk_noalloc: nbf %d exceeds the static scratch limit of %d", n,
                   HF_NOALLOC_MAX_NBF);
  hf_ctx* ctx = b->ctx;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (!b->have_work || b->work_tau != o.schwarz_tau || b->work_fp32 != o.fp32_bound ||
      b->work_rys != ((o.flags & HF_JK_RYS) != 0))
    return hf_fail(HF_ERR_INVALID,
                   "hf_fock_jk_noalloc: no quartet work lists for these options on this basis; call hf_fock_jk or "
                   "hf_count_quartets once with the same options first (that call allocates)");
  HF_CUDA(cudaSetDevice(ctx->device));
  double* scratch = nullptr;
  HF_CHECK(noalloc_scratch(ctx->device, &scratch));
  double* Jp = scratch;
  double* Kp = scratch + HF_NOALLOC_NN;
  int* counters = reinterpret_cast<int*>(scratch + 2 * HF_NOALLOC_NN);
  cudaStream_t st = ctx->stream;
  const size_t nn = (size_t)n * n;
  // the array keeps the previous call's contents: clear what starts at zero
  HF_CUDA(cudaMemsetAsync(Jp, 0, nn * sizeof(double), st));
  HF_CUDA(cudaMemsetAsync(Kp, 0, nn * sizeof(double), st));
  HF_CUDA(cudaMemsetAsync(counters, 0, sizeof(int) * 2 * HF_NCLASS, st));
  // the same class launches, precision tiers and symmetrisation as
  // hf_fock_jk, out of place from the static accumulators into J and K
  HF_CHECK(hf_jk_run(b, D, Jp, Kp, J, K, counters, o, st, nullptr, nullptr));
  HF_CUDA(cudaStreamSynchronize(st));
  return HF_OK;
}
