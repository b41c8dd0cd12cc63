// multi.cu -- multi-molecule J/K launches (batched SCF and serving).
#include <algorithm>
#include <cstdio>
#include <string>

#include "multi.h"

namespace {

// Zero J and K of every active molecule: blockIdx.y = molecule.
__global__ void zero_jk_batch(const MolJK* __restrict__ mols) {
  const MolJK m = mols[blockIdx.y];
  if (!m.active) return;
  const size_t nn = (size_t)m.nbf * m.nbf;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < nn; t += (size_t)gridDim.x * blockDim.x) {
    m.J[t] = 0.0;
    m.K[t] = 0.0;
    if (m.K2) m.K2[t] = 0.0;
  }
}

// J = 2 (J' + J'^T), K = K' + K'^T (and K2 likewise) in place for every
// active molecule.
__global__ void symmetrize_jk_batch(const MolJK* __restrict__ mols) {
  const MolJK m = mols[blockIdx.y];
  if (!m.active) return;
  const int n = m.nbf;
  const size_t nn = (size_t)n * n;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < nn; t += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(t / n), j = (int)(t % n);
    if (j < i) continue;
    const size_t ij = (size_t)i * n + j, ji = (size_t)j * n + i;
    const double sj = 2.0 * (m.J[ij] + m.J[ji]);
    m.J[ij] = sj;
    m.J[ji] = sj;
    const double sk = m.K[ij] + m.K[ji];
    m.K[ij] = sk;
    m.K[ji] = sk;
    if (m.K2) {
      const double s2 = m.K2[ij] + m.K2[ji];
      m.K2[ij] = s2;
      m.K2[ji] = s2;
    }
  }
}

}  // namespace

int MultiJK::build(hf_ctx* c, const std::vector<hf_basis*>& mols, const std::vector<const double*>& D,
                   const std::vector<double*>& J, const std::vector<double*>& K) {
  ctx = c;
  nmol = (int)mols.size();
  cudaStream_t st = ctx->stream;
  table_h.assign(nmol, MolJK{});
  mol_quartets.assign(nmol, 0);
  for (int m = 0; m < nmol; ++m) {
    hf_basis* b = mols[m];
    MolJK& t = table_h[m];
    t.D = D[m];
    t.J = J[m];
    t.K = K[m];
    t.nbf = b->nbf;
    t.active = 1;
    t.ps = hf_pairset(b);
    t.ketlist = b->ketlist.ptr;
    for (int y = 0; y < HF_NPAIRCLASS; ++y) t.ket_off[y] = b->class_begin[y];
  }
  HF_CHECK(table.alloc(ctx, std::max(nmol, 1)));
  if (nmol > 0)
    HF_CUDA(cudaMemcpyAsync(table.ptr, table_h.data(), sizeof(MolJK) * nmol, cudaMemcpyHostToDevice, st));
  HF_CHECK(counters.alloc(ctx, 2 * HF_NCLASS));
  std::vector<int> hb, hkb, hke, hio, hm, hs;
  for (int c2 = 0; c2 < 2 * HF_NCLASS; ++c2) {
    const int cls = c2 / 2, r = c2 % 2;
    hb.clear(); hkb.clear(); hke.clear(); hm.clear(); hs.clear(); hio.assign(1, 0);
    long long nq = 0;
    for (int m = 0; m < nmol; ++m) {
      const ClassWork& cw = r == 0 ? mols[m]->work64[cls] : mols[m]->work32[cls];
      for (size_t e = 0; e < cw.bra_h.size(); ++e) {
        const int cnt = cw.kend_h[e] - cw.kbeg_h[e];
        const int nsp = cw.nsplit_h.empty() ? 1 : cw.nsplit_h[e];
        // item offsets are int on the device: checked in 64 bits per entry
        const int chunk = cw.w.chunk > 0 ? cw.w.chunk : 1;
        const long long next = (long long)hio.back() + (long long)((cnt + chunk - 1) / chunk) * nsp;
        if (next > (1 << 30)) return hf_fail(HF_ERR_TOO_LARGE, "batched class %d: too many work items", cls);
        hb.push_back(cw.bra_h[e]);
        hkb.push_back(cw.kbeg_h[e]);
        hke.push_back(cw.kend_h[e]);
        hm.push_back(m);
        hs.push_back(nsp);
        hio.push_back((int)next);
        nq += cnt;
        mol_quartets[m] += cnt;
      }
    }
    const int nb = (int)hb.size();
    HF_CHECK(bra[c2].alloc(ctx, nb));
    HF_CHECK(kbeg[c2].alloc(ctx, nb));
    HF_CHECK(kend[c2].alloc(ctx, nb));
    HF_CHECK(mol[c2].alloc(ctx, nb));
    HF_CHECK(ioff[c2].alloc(ctx, nb + 1));
    HF_CHECK(nsplit[c2].alloc(ctx, nb));
    if (nb > 0) {
      HF_CUDA(cudaMemcpyAsync(nsplit[c2].ptr, hs.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, st));
      HF_CUDA(cudaMemcpyAsync(bra[c2].ptr, hb.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, st));
      HF_CUDA(cudaMemcpyAsync(kbeg[c2].ptr, hkb.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, st));
      HF_CUDA(cudaMemcpyAsync(kend[c2].ptr, hke.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, st));
      HF_CUDA(cudaMemcpyAsync(mol[c2].ptr, hm.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, st));
      HF_CUDA(cudaMemcpyAsync(ioff[c2].ptr, hio.data(), sizeof(int) * (nb + 1), cudaMemcpyHostToDevice, st));
    }
    JKWork& wk = w[c2];
    wk.bra = bra[c2].ptr;
    wk.ket = nullptr;
    wk.kbeg = kbeg[c2].ptr;
    wk.kend = kend[c2].ptr;
    wk.ioff = ioff[c2].ptr;
    wk.mol = mol[c2].ptr;
    wk.nsplit = nsplit[c2].ptr;
    wk.nbra = nb;
    wk.nitems = hio.back();
    wk.counter = counters.ptr + c2;
    // every molecule's lists were prepared with the same options
    wk.chunk = nmol > 0 ? (r == 0 ? mols[0]->work64[cls] : mols[0]->work32[cls]).w.chunk : ctx->ops[cls].chunk;
    wk.nchunk = nmol > 0 ? (r == 0 ? mols[0]->work64[cls] : mols[0]->work32[cls]).w.nchunk : 0;
    nquartets[c2] = nq;
    // the host vectors are reused for the next class: let the copies finish
    HF_CUDA(cudaStreamSynchronize(st));
  }
  return HF_OK;
}

int MultiJK::set_spin(int m, const double* Dj, const double* D2, double* K2) {
  if (m < 0 || m >= nmol) return hf_fail(HF_ERR_INVALID, "set_spin: molecule %d", m);
  table_h[m].Dj = Dj;
  table_h[m].D2 = D2;
  table_h[m].K2 = K2;
  HF_CUDA(cudaMemcpyAsync(table.ptr, table_h.data(), sizeof(MolJK) * nmol, cudaMemcpyHostToDevice, ctx->stream));
  HF_CUDA(cudaStreamSynchronize(ctx->stream));
  return HF_OK;
}

int MultiJK::set_active(const std::vector<int>& active) {
  for (int m = 0; m < nmol; ++m) table_h[m].active = active[m];
  if (nmol > 0) {
    HF_CUDA(cudaMemcpyAsync(table.ptr, table_h.data(), sizeof(MolJK) * nmol, cudaMemcpyHostToDevice, ctx->stream));
    HF_CUDA(cudaStreamSynchronize(ctx->stream));
  }
  return HF_OK;
}

int MultiJK::launch(const KernelCommon& kc, double* class_ms) {
  NvtxRange nv_build("multi-molecule J/K build");
  cudaStream_t st = ctx->stream;
  if (nmol == 0) return HF_OK;
  const dim3 g(std::max(1, 2 * ctx->num_sms / std::max(1, nmol)), nmol);
  zero_jk_batch<<<g, 256, 0, st>>>(table.ptr);
  HF_CUDA(cudaMemsetAsync(counters.ptr, 0, sizeof(int) * 2 * HF_NCLASS, st));
  const PairSet none{nullptr, nullptr, nullptr, nullptr};
  const MolJK one{};
  cudaEvent_t ev[2] = {nullptr, nullptr};
  if (class_ms) {
    HF_CUDA(cudaEventCreate(&ev[0]));
    HF_CUDA(cudaEventCreate(&ev[1]));
  }
  // Without per-class timing the class launches fork onto the side streams
  // (round robin, heaviest first) and join before the symmetrisation; the
  // classes share nothing but the J/K atomics, so they may run concurrently.
  const bool fork = class_ms == nullptr;
  if (fork) {
    HF_CUDA(cudaEventRecord(ctx->fork_ev, st));
    for (int k = 0; k < hf_ctx::kSide; ++k) HF_CUDA(cudaStreamWaitEvent(ctx->side[k], ctx->fork_ev, 0));
  }
  int nlaunch = 0;
  for (int cls = HF_NCLASS - 1; cls >= 0; --cls) {
    const EriClassOps& op = ctx->ops[cls];
    if (class_ms) HF_CUDA(cudaEventRecord(ev[0], st));
    bool any = false;
    for (int r = 0; r < 2; ++r) {
      const JKWork& wk = w[2 * cls + r];
      if (wk.nitems <= 0) continue;
      any = true;
      const int occ = std::max(r == 0 ? hf_occ_hi(op, jk_flags) : hf_occ_lo(op, jk_flags), 1);
      const LaunchShape sh = hf_launch_shape(ctx, occ, wk.nitems, grid_scale[cls]);
      cudaStream_t ls = fork ? ctx->side[nlaunch++ % hf_ctx::kSide] : st;
      NvtxRange nv_cls(op.name);
      (r == 0 ? hf_jk_hi(op, jk_flags) : hf_jk_lo(op, jk_flags))(wk, none, kc, one, table.ptr, sh.grid, sh.threads, ls);
    }
    if (class_ms && any) {
      HF_CUDA(cudaEventRecord(ev[1], st));
      HF_CUDA(cudaEventSynchronize(ev[1]));
      float ms = 0.f;
      HF_CUDA(cudaEventElapsedTime(&ms, ev[0], ev[1]));
      class_ms[cls] += ms;
    }
  }
  if (class_ms) {
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
  }
  HF_CUDA(cudaGetLastError());
  if (fork) {
    for (int k = 0; k < hf_ctx::kSide; ++k) {
      HF_CUDA(cudaEventRecord(ctx->join_ev[k], ctx->side[k]));
      HF_CUDA(cudaStreamWaitEvent(st, ctx->join_ev[k], 0));
    }
  }
  symmetrize_jk_batch<<<g, 256, 0, st>>>(table.ptr);
  HF_CUDA(cudaGetLastError());
  if (!capturing) HF_CHECK(hf_bounds_status(ctx, "multi-molecule J/K build"));
  return HF_OK;
}

int MultiJK::tune_step(const KernelCommon& kc) {
  static const int cand[3] = {0, 2, 1};
  for (int c = 0; c < HF_NCLASS; ++c) grid_scale[c] = cand[tune_iter];
  HF_CHECK(launch(kc, tune_ms[tune_iter]));
  if (++tune_iter == 3) {
    for (int c = 0; c < HF_NCLASS; ++c) {
      int best = 0;
      for (int k = 1; k < 3; ++k)
        if (tune_ms[k][c] > 0.0 && tune_ms[k][c] < tune_ms[best][c]) best = k;
      grid_scale[c] = cand[best];
    }
    tuned = true;
    // the choices, with the trial times, into the context's log
    std::string js = "{\"event\": \"autotune\", \"molecules\": " + std::to_string(nmol) + ", \"classes\": [";
    bool first = true;
    for (int c = 0; c < HF_NCLASS; ++c) {
      if (tune_ms[0][c] <= 0.0) continue;
      char buf[256];
      snprintf(buf, sizeof buf,
               "%s{\"class\": \"%s\", \"blocks_per_sm\": %d, \"ms_full\": %.4f, \"ms_2\": %.4f, \"ms_1\": %.4f}",
               first ? "" : ", ", ctx->ops[c].name, grid_scale[c], tune_ms[0][c], tune_ms[1][c], tune_ms[2][c]);
      js += buf;
      first = false;
    }
    js += "]}";
    hf_log_line(ctx, js.c_str());
  }
  return HF_OK;
}

int MultiJK::capture(const KernelCommon& kc) {
  cudaStream_t st = ctx->stream;
  if (graph_exec) {
    cudaGraphExecDestroy(graph_exec);
    graph_exec = nullptr;
  }
  if (graph) {
    cudaGraphDestroy(graph);
    graph = nullptr;
  }
  // make sure the occupancy queries are answered outside the capture
  for (int c = 0; c < HF_NCLASS; ++c) {
    ctx->ops[c].occ64();
    ctx->ops[c].occ32();
    ctx->ops[c].occdf();
    ctx->ops[c].occrys();
  }
  HF_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  capturing = true;
  const int rc = launch(kc);
  capturing = false;
  cudaGraph_t gph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(st, &gph);
  if (rc != HF_OK) {
    if (gph) cudaGraphDestroy(gph);
    return rc;
  }
  if (e != cudaSuccess) return hf_fail(HF_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
  graph = gph;
  HF_CUDA(cudaGraphInstantiate(&graph_exec, graph, 0));
  return HF_OK;
}

int MultiJK::run(const KernelCommon& kc) {
  if (!graph_exec) return launch(kc);
  HF_CUDA(cudaGraphLaunch(graph_exec, ctx->stream));
  HF_CHECK(hf_bounds_status(ctx, "multi-molecule J/K build"));
  return HF_OK;
}

MultiJK::~MultiJK() {
  if (graph_exec) cudaGraphExecDestroy(graph_exec);
  if (graph) cudaGraphDestroy(graph);
}
