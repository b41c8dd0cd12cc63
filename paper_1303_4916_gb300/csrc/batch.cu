// batch.cu -- many independent molecules solved together.
//
// Each SCF iteration: the per-molecule linear algebra (F' = X F X, syevd,
// D = C_occ C_occ^T) is enqueued for every active molecule, then ONE J/K
// launch per angular class covers the quartets of all molecules (MultiJK,
// replayed from a CUDA graph), then the per-molecule Fock/energy/DIIS
// updates are enqueued, with a single host synchronisation per iteration
// for all molecules.  Converged molecules drop out of the launches (their
// work items are skipped) and retire.  The first three iterations double
// as the autotuner's trials of the launch shape (blocks per SM) of each class.
#include <chrono>
#include <memory>
#include <vector>

#include "multi.h"
#include "scf_internal.h"

int scf_begin(hf_basis* b, ScfState& s, const hf_scf_opts& o, const double* G);
bool scf_after_iter(hf_basis* b, ScfState& s, const hf_scf_opts& o);
int scf_finish(hf_basis* b, ScfState& s, hf_scf_result* r);

extern "C" int hf_scf_solve_batch(hf_basis* const* bases, int count, const hf_scf_opts* opts, hf_scf_result* results,
                                  int* status) {
  if (!bases || !results || !status || count <= 0) return hf_fail(HF_ERR_INVALID, "hf_scf_solve_batch: bad arguments");
  hf_ctx* ctx = bases[0] ? bases[0]->ctx : nullptr;
  for (int i = 0; i < count; ++i)
    if (!bases[i] || bases[i]->ctx != ctx) return hf_fail(HF_ERR_INVALID, "basis %d missing or on another context", i);
  for (int i = 0; i < count; ++i)
    if (bases[i]->nelec % 2)
      return hf_fail(HF_ERR_ODD_ELECTRONS, "basis %d: closed-shell RHF needs an even electron count", i);
  hf_scf_opts o;
  hf_scf_opts_default(&o);
  if (opts) o = *opts;
  if (o.max_iter < 1 || o.diis_size < 0 || !(o.e_tol >= 0.0) || (o.flags & HF_SCF_STORED_ERI) || o.D0)
    return hf_fail(HF_ERR_INVALID, "hf_scf_solve_batch: bad options (stored ERI and D0 are single-molecule only)");
  HF_CHECK(hf_reject_deterministic(o.jk.flags, "hf_scf_solve_batch"));
  std::lock_guard<std::mutex> lk(ctx->mu);
  cudaSetDevice(ctx->device);
  const auto t0 = std::chrono::steady_clock::now();
  std::vector<std::unique_ptr<ScfState>> S(count);
  std::vector<int> active(count, 0);
  std::vector<hf_basis*> mols(bases, bases + count);
  std::vector<const double*> Dp(count);
  std::vector<double*> Jp(count), Kp(count);
  int first_error = HF_OK;
  for (int i = 0; i < count; ++i) {
    S[i].reset(new ScfState());
    int rc = hf_basis_prepare_work(mols[i], o.jk.schwarz_tau, o.jk.fp32_bound, o.jk.flags);
    if (rc == HF_OK) rc = scf_state_init(mols[i], *S[i], o.diis_size);
    if (rc == HF_OK) rc = scf_begin(mols[i], *S[i], o, nullptr);
    status[i] = rc;
    active[i] = rc == HF_OK;
    if (rc != HF_OK && first_error == HF_OK) first_error = rc;
    if (rc == HF_ERR_CUDA) return rc;
    Dp[i] = S[i]->D.ptr;
    Jp[i] = S[i]->J.ptr;
    Kp[i] = S[i]->K.ptr;
  }
  MultiJK mj;
  mj.jk_flags = o.jk.flags;
  HF_CHECK(mj.build(ctx, mols, Dp, Jp, Kp));
  HF_CHECK(mj.set_active(active));
  const KernelCommon kc = hf_kernel_common(ctx, o.jk.flags);
  bool tuned = false;
  int nactive = 0;
  for (int a : active) nactive += a;
  while (nactive > 0) {
    NvtxRange nv("scf iteration (batch)");
    for (int i = 0; i < count; ++i)
      if (active[i]) HF_CHECK(scf_density(mols[i], *S[i]));
    if (!mj.tuned) {
      HF_CHECK(mj.tune_step(kc));   // iterations 1-3 time the candidate launch shapes
    } else {
      if (!tuned) {
        HF_CHECK(mj.capture(kc));   // then the J/K phase is replayed from a graph
        tuned = true;
      }
      HF_CHECK(mj.run(kc));
    }
    for (int i = 0; i < count; ++i)
      if (active[i]) {
        S[i]->quartets += mj.mol_quartets[i];
        HF_CHECK(scf_post_jk(mols[i], *S[i]));
      }
    HF_CUDA(cudaStreamSynchronize(ctx->stream));
    bool changed = false;
    for (int i = 0; i < count; ++i) {
      if (!active[i]) continue;
      HF_CHECK(scf_diis_step(mols[i], *S[i]));
      const bool done = scf_after_iter(mols[i], *S[i], o);
      hf_log_scf_iter(ctx, "batch", (unsigned long long)i, mols[i]->nbf, S[i]->iter, S[i]->energy, S[i]->delta_e,
                      S[i]->diis_error, std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(),
                      S[i]->converged);
      if (done) {
        HF_CHECK(scf_finish(mols[i], *S[i], &results[i]));
        status[i] = S[i]->converged ? HF_OK : HF_ERR_NOT_CONVERGED;
        if (!S[i]->converged && first_error == HF_OK) first_error = HF_ERR_NOT_CONVERGED;
        active[i] = 0;
        --nactive;
        changed = true;
      }
    }
    if (changed) HF_CHECK(mj.set_active(active));
  }
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  for (int i = 0; i < count; ++i) results[i].seconds = secs;
  if (first_error != HF_OK) return hf_fail(first_error, "hf_scf_solve_batch: at least one molecule failed (see status)");
  return HF_OK;
}
