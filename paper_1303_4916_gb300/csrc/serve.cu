// serve.cu -- continuous-batching SCF serving loop.
//
// A worker thread owns the GPU work of the server.  Requests wait in a FIFO
// queue; at every iteration boundary the worker admits requests from the
// head of the queue while fewer than max_active are in flight and their
// estimated device footprint (pair data, work lists, SCF state with the
// DIIS history) fits the HBM budget.  All active molecules advance one SCF
// iteration per round together: per-molecule linear algebra, then one J/K
// launch per angular class over the quartets of all of them (MultiJK), then
// the per-molecule Fock/energy/DIIS updates with one host synchronisation.
// Converged (or failed) molecules retire at the end of the round, freeing
// their slot and memory; new arrivals join at the next round.  Every wait
// of the worker and of hf_serve_drain is bounded.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <thread>
#include <unordered_map>
#include <vector>

#include "multi.h"
#include "scf_internal.h"

namespace {

enum ReqState { QUEUED = 0, ACTIVE = 1, DONE = 2 };

struct Request {
  uint64_t ticket = 0;
  std::vector<hf_atom> atoms;
  std::vector<hf_shell> shells;
  std::vector<double> exps, coefs;
  int nelec = 0;
  size_t footprint = 0;
  ReqState state = QUEUED;
  hf_serve_result result{};
  // while active
  hf_basis* basis = nullptr;
  std::unique_ptr<ScfState> scf;
};

int ncart(int l) { return (l + 1) * (l + 2) / 2; }

// Device bytes an admitted request holds: primitive-pair records (FP64 80 B,
// FP32 48 B and df64 80 B per primitive pair), shell-pair info and ket
// lists, work lists (bounded by the bucket count per pair), SCF state: 12
// n^2 matrices plus two for the syevd workspace and host-pointer staging,
// DIIS 2 m n^2, plus 10%.
size_t estimate_footprint(const hf_request* r, int diis) {
  long long nbf = 0, npp = 0, np = 0;
  for (int s = 0; s < r->nshell; ++s) nbf += ncart(r->shells[s].l);
  for (int a = 0; a < r->nshell; ++a)
    for (int b = 0; b <= a; ++b) {
      npp += (long long)r->shells[a].nprim * r->shells[b].nprim;
      ++np;
    }
  const double n2 = (double)nbf * nbf * 8.0;
  double bytes = npp * 208.0 + np * 64.0 + np * 2.0 * 16.0 * 4.0 * 6.0 + (14.0 + 2.0 * diis) * n2;
  return (size_t)(1.1 * bytes) + (1u << 20);
}

}  // namespace

struct hf_server {
  hf_ctx* ctx = nullptr;
  hf_serve_opts opts{};
  size_t budget = 0, used = 0;
  std::mutex mu;
  std::condition_variable cv;       // wakes the worker
  std::condition_variable done_cv;  // wakes drain()
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;
  std::vector<Request*> active;
  uint64_t next_ticket = 1;
  bool stop = false;
  std::thread worker;
  std::chrono::steady_clock::time_point t0;
  int grid_scale[HF_NCLASS] = {};
  bool tuned = false;
  int worker_error = HF_OK;

  double now() const { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); }
  void run();
  void retire(Request* r, int status);
};

void hf_server::retire(Request* r, int status) {
  // caller holds mu
  r->result.status = status;
  r->result.t_done = now();
  if (r->scf) {
    r->result.fock_builds = r->scf->fock_builds;
    r->result.quartets = r->scf->quartets;
  }
  r->scf.reset();
  if (r->basis) {
    hf_basis_destroy(r->basis);
    r->basis = nullptr;
  }
  used -= std::min(used, r->footprint);
  r->state = DONE;
}

void hf_server::run() {
  cudaSetDevice(ctx->device);
  const KernelCommon kc = hf_kernel_common(ctx, opts.scf.jk.flags);
  std::unique_ptr<MultiJK> mj;
  bool membership_changed = true;
  for (;;) {
    std::vector<Request*> admitted;
    {
      std::unique_lock<std::mutex> lk(mu);
      for (;;) {
        while (!queue.empty() && (int)active.size() + (int)admitted.size() < opts.max_active) {
          Request* r = reqs[queue.front()].get();
          if (used + r->footprint > budget && !(active.empty() && admitted.empty())) break;
          queue.pop_front();
          used += r->footprint;
          r->state = ACTIVE;
          r->result.t_admit = now();
          admitted.push_back(r);
        }
        if (!admitted.empty() || !active.empty()) break;
        if (stop) return;
        cv.wait_for(lk, std::chrono::milliseconds(50));
      }
    }
    // set up the newly admitted molecules (outside the lock: GPU work)
    std::lock_guard<std::mutex> glk(ctx->mu);
    for (Request* r : admitted) {
      int rc = hf_basis_create(ctx, r->atoms.data(), (int)r->atoms.size(), r->shells.data(), (int)r->shells.size(),
                               r->exps.data(), r->coefs.data(), r->nelec, &r->basis);
      r->scf.reset(new ScfState());
      if (rc == HF_OK) rc = hf_basis_prepare_work(r->basis, opts.scf.jk.schwarz_tau, opts.scf.jk.fp32_bound, opts.scf.jk.flags);
      if (rc == HF_OK) rc = scf_state_init(r->basis, *r->scf, opts.scf.diis_size);
      if (rc == HF_OK) rc = scf_begin(r->basis, *r->scf, opts.scf, nullptr);
      std::lock_guard<std::mutex> lk(mu);
      if (rc != HF_OK) {
        retire(r, rc);
        done_cv.notify_all();
      } else {
        r->result.nbf = r->basis->nbf;
        active.push_back(r);
        membership_changed = true;
      }
    }
    if (active.empty()) continue;
    int rc = HF_OK;
    if (membership_changed) {
      mj.reset(new MultiJK());
      mj->jk_flags = opts.scf.jk.flags;
      std::vector<hf_basis*> mols;
      std::vector<const double*> Dp;
      std::vector<double*> Jp, Kp;
      for (Request* r : active) {
        mols.push_back(r->basis);
        Dp.push_back(r->scf->D.ptr);
        Jp.push_back(r->scf->J.ptr);
        Kp.push_back(r->scf->K.ptr);
      }
      rc = mj->build(ctx, mols, Dp, Jp, Kp);
      if (tuned)
        for (int c = 0; c < HF_NCLASS; ++c) mj->grid_scale[c] = grid_scale[c];
      membership_changed = false;
    }
    // one SCF iteration for every active molecule
    NvtxRange nv("serve round");
    for (Request* r : active)
      if (rc == HF_OK) rc = scf_density(r->basis, *r->scf);
    if (rc == HF_OK && !tuned) {
      rc = mj->tune_step(kc);       // the first rounds double as autotuner trials
      if (mj->tuned) {
        for (int c = 0; c < HF_NCLASS; ++c) grid_scale[c] = mj->grid_scale[c];
        tuned = true;
      }
    } else if (rc == HF_OK) {
      rc = mj->launch(kc);
    }
    for (size_t i = 0; i < active.size() && rc == HF_OK; ++i) {
      active[i]->scf->quartets += mj->mol_quartets[i];
      rc = scf_post_jk(active[i]->basis, *active[i]->scf);
    }
    if (rc == HF_OK && cudaStreamSynchronize(ctx->stream) != cudaSuccess) rc = hf_fail(HF_ERR_CUDA, "serve sync");
    std::vector<Request*> keep;
    std::vector<std::pair<Request*, int>> finished;
    for (Request* r : active) {
      if (rc != HF_OK) {
        finished.push_back({r, rc});
        continue;
      }
      int rr = scf_diis_step(r->basis, *r->scf);
      if (rr != HF_OK) {
        finished.push_back({r, rr});
        continue;
      }
      const bool done = scf_after_iter(r->basis, *r->scf, opts.scf);
      hf_log_scf_iter(ctx, "serve", (unsigned long long)r->ticket, r->basis->nbf, r->scf->iter, r->scf->energy,
                      r->scf->delta_e, r->scf->diis_error, now() - r->result.t_admit, r->scf->converged);
      if (done) {
        hf_scf_result res{};
        scf_finish(r->basis, *r->scf, &res);
        r->result.energy = res.energy;
        r->result.iterations = res.iterations;
        r->result.converged = res.converged;
        finished.push_back({r, res.converged ? HF_OK : HF_ERR_NOT_CONVERGED});
      } else {
        keep.push_back(r);
      }
    }
    if (!finished.empty()) {
      std::lock_guard<std::mutex> lk(mu);
      for (auto& f : finished) retire(f.first, f.second);
      active = keep;
      membership_changed = true;
      if (rc != HF_OK) worker_error = rc;
      done_cv.notify_all();
    }
  }
}

extern "C" void hf_serve_opts_default(hf_serve_opts* o) {
  if (!o) return;
  o->max_active = 64;
  o->queue_capacity = 100000;
  o->hbm_budget = 0;
  hf_scf_opts_default(&o->scf);
}

extern "C" int hf_serve_create(hf_ctx* ctx, const hf_serve_opts* opts, hf_server** out) {
  if (!out) return hf_fail(HF_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!ctx) return hf_fail(HF_ERR_INVALID, "null context");
  hf_serve_opts o;
  hf_serve_opts_default(&o);
  if (opts) o = *opts;
  if (o.max_active < 1 || o.queue_capacity < 1 || o.scf.max_iter < 1 || o.scf.diis_size < 0 ||
      (o.scf.flags & HF_SCF_STORED_ERI) || o.scf.D0)
    return hf_fail(HF_ERR_INVALID, "hf_serve_create: bad options");
  HF_CHECK(hf_reject_deterministic(o.scf.jk.flags, "hf_serve_create"));
  hf_server* s = new (std::nothrow) hf_server();
  if (!s) return hf_fail(HF_ERR_OOM, "host allocation");
  s->ctx = ctx;
  s->opts = o;
  s->budget = o.hbm_budget ? o.hbm_budget : ctx->hbm_budget;
  s->t0 = std::chrono::steady_clock::now();
  ctx->live_bases.fetch_add(1);
  s->worker = std::thread([s] { s->run(); });
  *out = s;
  return HF_OK;
}

extern "C" int hf_serve_submit(hf_server* s, const hf_request* req, uint64_t* ticket) {
  if (!s || !req || !ticket) return hf_fail(HF_ERR_INVALID, "hf_serve_submit: null argument");
  if (!req->atoms || !req->shells || !req->exps || !req->coefs || req->natom <= 0 || req->nshell <= 0 ||
      req->nprim <= 0)
    return hf_fail(HF_ERR_INVALID, "hf_serve_submit: empty request");
  if (req->n_electrons < 0 || req->n_electrons % 2)
    return hf_fail(HF_ERR_ODD_ELECTRONS, "hf_serve_submit: electron count %d", req->n_electrons);
  for (int k = 0; k < req->nshell; ++k) {
    const hf_shell& sh = req->shells[k];
    if (sh.l < 0 || sh.atom < 0 || sh.atom >= req->natom || sh.nprim < 1 || sh.prim_off < 0 ||
        sh.prim_off + sh.nprim > req->nprim)
      return hf_fail(HF_ERR_INVALID, "hf_serve_submit: shell %d out of range", k);
    if (sh.l > HF_LMAX) return hf_fail(HF_ERR_UNSUPPORTED_L, "hf_serve_submit: shell %d l=%d", k, sh.l);
  }
  std::unique_ptr<Request> r(new (std::nothrow) Request());
  if (!r) return hf_fail(HF_ERR_OOM, "host allocation");
  r->atoms.assign(req->atoms, req->atoms + req->natom);
  r->shells.assign(req->shells, req->shells + req->nshell);
  r->exps.assign(req->exps, req->exps + req->nprim);
  r->coefs.assign(req->coefs, req->coefs + req->nprim);
  r->nelec = req->n_electrons;
  r->footprint = estimate_footprint(req, s->opts.scf.diis_size);
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) return hf_fail(HF_ERR_CANCELLED, "server is shutting down");
  if (r->footprint > s->budget)
    return hf_fail(HF_ERR_TOO_LARGE, "request needs ~%zu bytes, budget %zu", r->footprint, s->budget);
  if ((int)s->queue.size() >= s->opts.queue_capacity) return hf_fail(HF_ERR_QUEUE_FULL, "queue at capacity");
  r->ticket = s->next_ticket++;
  r->result.t_submit = s->now();
  r->result.status = HF_PENDING;
  *ticket = r->ticket;
  s->queue.push_back(r->ticket);
  s->reqs[r->ticket] = std::move(r);
  s->cv.notify_one();
  return HF_OK;
}

extern "C" int hf_serve_poll(hf_server* s, uint64_t ticket, hf_serve_result* result) {
  if (!s) return hf_fail(HF_ERR_INVALID, "null server");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return HF_ERR_NOT_FOUND;
  if (it->second->state != DONE) return HF_PENDING;
  if (result) *result = it->second->result;
  s->reqs.erase(it);
  return HF_OK;
}

extern "C" int hf_serve_cancel(hf_server* s, uint64_t ticket) {
  if (!s) return hf_fail(HF_ERR_INVALID, "null server");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end() || it->second->state != QUEUED) return HF_ERR_NOT_FOUND;
  s->queue.erase(std::remove(s->queue.begin(), s->queue.end(), ticket), s->queue.end());
  s->reqs.erase(it);
  s->done_cv.notify_all();
  return HF_OK;
}

extern "C" double hf_serve_now(hf_server* s) { return s ? s->now() : 0.0; }

extern "C" int hf_serve_drain(hf_server* s, double timeout_s) {
  if (!s) return hf_fail(HF_ERR_INVALID, "null server");
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    bool busy = !s->queue.empty() || !s->active.empty();
    if (!busy) {
      for (auto& kv : s->reqs)
        if (kv.second->state != DONE) { busy = true; break; }
    }
    if (!busy) return s->worker_error == HF_OK ? HF_OK : s->worker_error;
    if (std::chrono::steady_clock::now() >= deadline) return hf_fail(HF_ERR_TIMEOUT, "drain timed out");
    s->done_cv.wait_for(lk, std::chrono::milliseconds(20));
  }
}

extern "C" void hf_serve_destroy(hf_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    // queued requests are dropped; active ones finish their solve first
    for (uint64_t t : s->queue) s->reqs.erase(t);
    s->queue.clear();
  }
  s->cv.notify_all();
  if (s->worker.joinable()) s->worker.join();
  for (auto& kv : s->reqs) {
    if (kv.second->basis) hf_basis_destroy(kv.second->basis);
  }
  hf_ctx* ctx = s->ctx;
  delete s;
  // a server keeps its context alive like a basis does
  if (ctx->live_bases.fetch_sub(1) == 1 && ctx->destroy_pending.load()) hf_ctx_teardown(ctx);
}
