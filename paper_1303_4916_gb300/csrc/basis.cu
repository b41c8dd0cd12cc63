// basis.cu -- basis construction, shell-pair data, Schwarz factors,
// quartet bucketing, the J/K launch sequence, one-electron integrals and the
// stored-tensor path.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "eri.cuh"
#include "hf_internal.h"

static const double kPi = 3.14159265358979323846;

// Primitive pairs whose magnitude bound is below this are skipped; their
// contribution to any integral is below ~1e-16.
static const double kPrimEps = 1e-17;

static double dfact(int n) {
  double r = 1.0;
  for (int k = n; k > 1; k -= 2) r *= k;
  return r;
}

static int ncart(int l) { return (l + 1) * (l + 2) / 2; }

// ------------------------------------------------------------- pair kernel
// One thread per shell pair (A, B), l_A >= l_B: for each primitive pair
// p = a + b, P = (a A + b B)/p, PA = P - A and
// K = c_a c_b exp(-ab/p |AB|^2) sqrt(2) pi^(5/4) / p and the exponent a of
// A's primitive (the derivative integrals need it); records are sorted by
// the magnitude bound |K| (2p)^(-1/4) (1 + |AB| + p^(-1/2))^(l_A+l_B) and
// those below kPrimEps are not counted.
__global__ void pair_kernel(int npairs, const int* __restrict__ pA, const int* __restrict__ pB,
                            const int* __restrict__ poff, const double* __restrict__ sh_xyz,
                            const int* __restrict__ sh_l, const int* __restrict__ sh_nprim,
                            const int* __restrict__ sh_prim, const int* __restrict__ sh_bf,
                            const double* __restrict__ exps, const double* __restrict__ coefs,
                            double* __restrict__ prim64, float* __restrict__ prim32, float* __restrict__ primdf,
                            PairInfo* __restrict__ info, double eps) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= npairs) return;
  const int A = pA[t], B = pB[t];
  const double Ax = sh_xyz[3 * A], Ay = sh_xyz[3 * A + 1], Az = sh_xyz[3 * A + 2];
  const double Bx = sh_xyz[3 * B], By = sh_xyz[3 * B + 1], Bz = sh_xyz[3 * B + 2];
  const double ABx = Ax - Bx, ABy = Ay - By, ABz = Az - Bz;
  const double r2 = ABx * ABx + ABy * ABy + ABz * ABz;
  const double rab = sqrt(r2);
  const int KA = sh_nprim[A], KB = sh_nprim[B], l = sh_l[A] + sh_l[B];
  const int n = KA * KB;
  double mag[HF_MAX_NPRIM * HF_MAX_NPRIM];
  int order[HF_MAX_NPRIM * HF_MAX_NPRIM];
  for (int k = 0; k < n; ++k) {
    const double a = exps[sh_prim[A] + k / KB], b = exps[sh_prim[B] + k % KB];
    const double p = a + b;
    const double K = coefs[sh_prim[A] + k / KB] * coefs[sh_prim[B] + k % KB] * exp(-a * b / p * r2) * 1.4142135623730951 *
                     pow(kPi, 1.25) / p;
    mag[k] = fabs(K) * pow(2.0 * p, -0.25) * pow(1.0 + rab + 1.0 / sqrt(p), (double)l);
    order[k] = k;
  }
  for (int i = 1; i < n; ++i) {  // insertion sort, descending magnitude
    const int o = order[i];
    int j = i - 1;
    while (j >= 0 && mag[order[j]] < mag[o]) {
      order[j + 1] = order[j];
      --j;
    }
    order[j + 1] = o;
  }
  int nsig = 0;
  const int base = poff[t];
  for (int s = 0; s < n; ++s) {
    const int k = order[s];
    if (mag[k] >= eps) ++nsig;
    const double a = exps[sh_prim[A] + k / KB], b = exps[sh_prim[B] + k % KB];
    const double p = a + b;
    const double K = coefs[sh_prim[A] + k / KB] * coefs[sh_prim[B] + k % KB] * exp(-a * b / p * r2) * 1.4142135623730951 *
                     pow(kPi, 1.25) / p;
    const double Px = (a * Ax + b * Bx) / p, Py = (a * Ay + b * By) / p, Pz = (a * Az + b * Bz) / p;
    double* r = prim64 + (size_t)(base + s) * PRIM64_STRIDE;
    r[0] = p; r[1] = 0.5 / p; r[2] = Px; r[3] = Py; r[4] = Pz;
    r[5] = Px - Ax; r[6] = Py - Ay; r[7] = Pz - Az; r[8] = K; r[9] = a;
    float* f = prim32 + (size_t)(base + s) * PRIM32_STRIDE;
    for (int x = 0; x < 10; ++x) f[x] = (float)r[x];
    f[10] = 0.f; f[11] = 0.f;
    float* g = primdf + (size_t)(base + s) * PRIMDF_STRIDE;
    for (int x = 0; x < 10; ++x) {
      const float h = __double2float_rn(r[x]);
      g[2 * x] = h;
      g[2 * x + 1] = __double2float_rn(r[x] - (double)h);
    }
  }
  PairInfo pi;
  pi.bfA = sh_bf[A];
  pi.bfB = sh_bf[B];
  pi.prim0 = base;
  pi.nprim = nsig;
  pi.AB[0] = ABx; pi.AB[1] = ABy; pi.AB[2] = ABz;
  pi.same = (A == B);
  pi.pad = 0;
  info[t] = pi;
}

// ------------------------------------------------------------- symmetrise
// J = 2 (J' + J'^T), K = K' + K'^T (and K2 = K2' + K2'^T when K2 is given),
// from the accumulators into (J, K, K2).  In place when the accumulators
// are the outputs: each unordered pair {i, j} is read and written by one
// thread only, so the two forms share this kernel.
__global__ void symmetrize_jk(const double* Jp, const double* Kp, double* J, double* K, const double* K2p, double* K2,
                              int n) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long tot = (long long)n * n;
  if (t >= tot) return;
  const int i = (int)(t / n), j = (int)(t % n);
  if (j < i) return;
  const size_t ij = (size_t)i * n + j, ji = (size_t)j * n + i;
  const double sj = 2.0 * (Jp[ij] + Jp[ji]);
  const double sk = Kp[ij] + Kp[ji];
  J[ij] = sj;
  J[ji] = sj;
  K[ij] = sk;
  K[ji] = sk;
  if (K2) {
    const double s2 = K2p[ij] + K2p[ji];
    K2[ij] = s2;
    K2[ji] = s2;
  }
}

// J = 2 (J' + J'^T), K = K' + K'^T (K2 likewise when given) from fixed-point
// accumulators (two 64-bit words per element, units 2^-20 and 2^-56).
__device__ __forceinline__ double fixed_value(const unsigned long long* q, size_t i) {
  return (double)(long long)q[2 * i] * (1.0 / 1048576.0) + (double)(long long)q[2 * i + 1] * 0x1p-56;
}
__global__ void finish_fixed(const unsigned long long* __restrict__ Jq, const unsigned long long* __restrict__ Kq,
                             const unsigned long long* __restrict__ K2q, double* __restrict__ J,
                             double* __restrict__ K, double* __restrict__ K2, int n) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)n * n) return;
  const int i = (int)(t / n), j = (int)(t % n);
  if (j < i) return;
  const size_t ij = (size_t)i * n + j, ji = (size_t)j * n + i;
  const double sj = 2.0 * (fixed_value(Jq, ij) + fixed_value(Jq, ji));
  const double sk = fixed_value(Kq, ij) + fixed_value(Kq, ji);
  J[ij] = sj;
  J[ji] = sj;
  K[ij] = sk;
  K[ji] = sk;
  if (K2) {
    const double s2 = fixed_value(K2q, ij) + fixed_value(K2q, ji);
    K2[ij] = s2;
    K2[ji] = s2;
  }
}

// ------------------------------------------------------------- basis create
extern "C" int hf_basis_create(hf_ctx* ctx, const hf_atom* atoms, int natom, const hf_shell* shells, int nshell,
                               const double* exps, const double* coefs, int n_electrons, hf_basis** out) {
  if (!out) return hf_fail(HF_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!ctx || !atoms || !shells || !exps || !coefs || natom <= 0 || nshell <= 0)
    return hf_fail(HF_ERR_INVALID, "hf_basis_create: null or empty input");
  if (n_electrons < 0) return hf_fail(HF_ERR_INVALID, "negative electron count");
  int nprim = 0, nbf = 0, lmax = 0;
  for (int s = 0; s < nshell; ++s) {
    const hf_shell& sh = shells[s];
    if (sh.l < 0) return hf_fail(HF_ERR_INVALID, "shell %d: negative l", s);
    if (sh.l > HF_LMAX) return hf_fail(HF_ERR_UNSUPPORTED_L, "shell %d: l = %d above %d", s, sh.l, HF_LMAX);
    if (sh.atom < 0 || sh.atom >= natom) return hf_fail(HF_ERR_INVALID, "shell %d: atom index %d", s, sh.atom);
    if (sh.nprim < 1 || sh.nprim > HF_MAX_NPRIM) return hf_fail(HF_ERR_INVALID, "shell %d: nprim %d", s, sh.nprim);
    if (sh.prim_off < 0) return hf_fail(HF_ERR_INVALID, "shell %d: prim_off", s);
    nprim = std::max(nprim, sh.prim_off + sh.nprim);
    nbf += ncart(sh.l);
    lmax = std::max(lmax, sh.l);
  }
  for (int k = 0; k < nprim; ++k)
    if (!(exps[k] > 0.0) || !std::isfinite(exps[k]) || !std::isfinite(coefs[k]))
      return hf_fail(HF_ERR_INVALID, "primitive %d: exponent must be positive and finite", k);
  for (int a = 0; a < natom; ++a)
    for (int x = 0; x < 3; ++x)
      if (!std::isfinite(atoms[a].xyz[x])) return hf_fail(HF_ERR_INVALID, "atom %d: non-finite coordinate", a);

  cudaSetDevice(ctx->device);
  if (ctx->destroy_pending.load()) return hf_fail(HF_ERR_INVALID, "hf_basis_create: context is being destroyed");
  hf_basis* b = new (std::nothrow) hf_basis();
  if (!b) return hf_fail(HF_ERR_OOM, "host allocation");
  b->ctx = ctx;
  ctx->live_bases.fetch_add(1);
  b->natom = natom;
  b->nshell = nshell;
  b->nbf = nbf;
  b->nprim = nprim;
  b->nelec = n_electrons;
  b->lmax = lmax;
  b->atoms.assign(atoms, atoms + natom);
  b->sh_atom.resize(nshell);
  b->sh_l.resize(nshell);
  b->sh_nprim.resize(nshell);
  b->sh_prim.resize(nshell);
  b->sh_bf.resize(nshell + 1);
  b->exps.assign(exps, exps + nprim);
  b->coefs.assign(nprim, 0.0);
  int bf = 0;
  for (int s = 0; s < nshell; ++s) {
    b->sh_atom[s] = shells[s].atom;
    b->sh_l[s] = shells[s].l;
    b->sh_nprim[s] = shells[s].nprim;
    b->sh_prim[s] = shells[s].prim_off;
    b->sh_bf[s] = bf;
    bf += ncart(shells[s].l);
  }
  b->sh_bf[nshell] = bf;
  // Contracted normalisation (Eq. 1 functions of unit norm): primitive
  // factors for the axial component x^l, then the contraction rescaled by
  // its self-overlap.  Other Cartesian components carry comp_scale().
  for (int s = 0; s < nshell; ++s) {
    const int l = b->sh_l[s], K = b->sh_nprim[s], p0 = b->sh_prim[s];
    std::vector<double> c(K);
    for (int k = 0; k < K; ++k) {
      const double a = exps[p0 + k];
      c[k] = coefs[p0 + k] * pow(2.0 * a / kPi, 0.75) * pow(4.0 * a, 0.5 * l) / sqrt(dfact(2 * l - 1));
    }
    double self = 0.0;
    for (int i = 0; i < K; ++i)
      for (int j = 0; j < K; ++j) {
        const double p = exps[p0 + i] + exps[p0 + j];
        self += c[i] * c[j] * pow(kPi / p, 1.5) * dfact(2 * l - 1) / pow(2.0 * p, l);
      }
    if (!(self > 0.0)) {
      delete b;
      return hf_fail(HF_ERR_INVALID, "shell %d: contraction has zero norm", s);
    }
    for (int k = 0; k < K; ++k) b->coefs[p0 + k] = c[k] / sqrt(self);
  }
  double en = 0.0;
  for (int i = 0; i < natom; ++i)
    for (int j = 0; j < i; ++j) {
      double r2 = 0.0;
      for (int x = 0; x < 3; ++x) {
        const double d = atoms[i].xyz[x] - atoms[j].xyz[x];
        r2 += d * d;
      }
      if (r2 == 0.0 && atoms[i].Z != 0 && atoms[j].Z != 0) {
        delete b;
        return hf_fail(HF_ERR_INVALID, "atoms %d and %d coincide", i, j);
      }
      if (r2 > 0.0) en += (double)atoms[i].Z * atoms[j].Z / sqrt(r2);
    }
  b->e_nuc = en;

  // Shell pairs, grouped by pair class; within a pair l_A >= l_B.
  std::vector<int> cls_of;
  for (int i = 0; i < nshell; ++i)
    for (int j = 0; j <= i; ++j) {
      int A = i, B = j;
      if (b->sh_l[B] > b->sh_l[A]) std::swap(A, B);
      b->pair_A.push_back(A);
      b->pair_B.push_back(B);
      cls_of.push_back(pair_class(b->sh_l[A], b->sh_l[B]));
    }
  const int np = (int)b->pair_A.size();
  std::vector<int> idx(np);
  std::iota(idx.begin(), idx.end(), 0);
  std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return cls_of[x] < cls_of[y]; });
  std::vector<int> pA(np), pB(np), poff(np);
  int off = 0;
  {
    int cnt[HF_NPAIRCLASS] = {};
    for (int k = 0; k < np; ++k) ++cnt[cls_of[k]];
    b->class_begin[0] = 0;
    for (int c = 0; c < HF_NPAIRCLASS; ++c) b->class_begin[c + 1] = b->class_begin[c] + cnt[c];
  }
  for (int k = 0; k < np; ++k) {
    pA[k] = b->pair_A[idx[k]];
    pB[k] = b->pair_B[idx[k]];
    poff[k] = off;
    off += b->sh_nprim[pA[k]] * b->sh_nprim[pB[k]];
  }
  b->pair_A = pA;
  b->pair_B = pB;
  b->npairs = np;
  b->nprimpairs = off;

  int rc = HF_OK;
  std::vector<double> sh_xyz(3 * nshell);
  for (int s = 0; s < nshell; ++s)
    for (int x = 0; x < 3; ++x) sh_xyz[3 * s + x] = atoms[b->sh_atom[s]].xyz[x];
  DevArray<int> dA, dB, dOff, dl, dn, dp, dbf;
  DevArray<double> dxyz, dexp, dcoef;
  cudaStream_t st = ctx->stream;
  do {
    if ((rc = dA.alloc(ctx, np)) || (rc = dB.alloc(ctx, np)) || (rc = dOff.alloc(ctx, np)) ||
        (rc = dl.alloc(ctx, nshell)) || (rc = dn.alloc(ctx, nshell)) || (rc = dp.alloc(ctx, nshell)) ||
        (rc = dbf.alloc(ctx, nshell + 1)) || (rc = dxyz.alloc(ctx, 3 * nshell)) || (rc = dexp.alloc(ctx, nprim)) ||
        (rc = dcoef.alloc(ctx, nprim)) || (rc = b->prim64.alloc(ctx, (size_t)off * PRIM64_STRIDE)) ||
        (rc = b->prim32.alloc(ctx, (size_t)off * PRIM32_STRIDE)) ||
        (rc = b->primdf.alloc(ctx, (size_t)off * PRIMDF_STRIDE)) || (rc = b->pinfo.alloc(ctx, np)) ||
        (rc = b->Q.alloc(ctx, np)) || (rc = b->ketlist.alloc(ctx, np)) || (rc = b->counters.alloc(ctx, 2 * HF_NCLASS)))
      break;
#define UP(dst, src, cnt)                                                                                      \
  if (cudaMemcpyAsync(dst.ptr, src, sizeof(*dst.ptr) * (cnt), cudaMemcpyHostToDevice, st) != cudaSuccess) { \
    rc = hf_fail(HF_ERR_CUDA, "upload");                                                                     \
    break;                                                                                                   \
  }
    UP(dA, pA.data(), np);
    UP(dB, pB.data(), np);
    UP(dOff, poff.data(), np);
    UP(dl, b->sh_l.data(), nshell);
    UP(dn, b->sh_nprim.data(), nshell);
    UP(dp, b->sh_prim.data(), nshell);
    UP(dbf, b->sh_bf.data(), nshell + 1);
    UP(dxyz, sh_xyz.data(), 3 * nshell);
    UP(dexp, b->exps.data(), nprim);
    UP(dcoef, b->coefs.data(), nprim);
#undef UP
    pair_kernel<<<(np + 127) / 128, 128, 0, st>>>(np, dA.ptr, dB.ptr, dOff.ptr, dxyz.ptr, dl.ptr, dn.ptr, dp.ptr, dbf.ptr,
                                                  dexp.ptr, dcoef.ptr, b->prim64.ptr, b->prim32.ptr, b->primdf.ptr,
                                                  b->pinfo.ptr, kPrimEps);
    if (cudaGetLastError() != cudaSuccess) { rc = hf_fail(HF_ERR_CUDA, "pair_kernel launch"); break; }
    // Schwarz factors per pair class, using the (X|X) diagonal quartets.
    DevArray<int> ids;
    if ((rc = ids.alloc(ctx, np))) break;
    std::vector<int> iota_h(np);
    std::iota(iota_h.begin(), iota_h.end(), 0);
    if (cudaMemcpyAsync(ids.ptr, iota_h.data(), sizeof(int) * np, cudaMemcpyHostToDevice, st) != cudaSuccess) {
      rc = hf_fail(HF_ERR_CUDA, "upload");
      break;
    }
    const PairSet ps = hf_pairset(b);
    const KernelCommon kc = hf_kernel_common(ctx, 0);
    for (int X = 0; X < HF_NPAIRCLASS; ++X) {
      const int n = b->class_begin[X + 1] - b->class_begin[X];
      if (n <= 0) continue;
      ctx->ops[X * (X + 1) / 2 + X].schwarz(ids.ptr + b->class_begin[X], n, ps, kc, b->Q.ptr, st);
    }
    if (cudaGetLastError() != cudaSuccess) { rc = hf_fail(HF_ERR_CUDA, "schwarz launch"); break; }
    b->Q_h.resize(np);
    std::vector<PairInfo> info_h(np);
    if (cudaMemcpyAsync(b->Q_h.data(), b->Q.ptr, sizeof(double) * np, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(info_h.data(), b->pinfo.ptr, sizeof(PairInfo) * np, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      rc = hf_fail(HF_ERR_CUDA, "pair setup: %s", cudaGetErrorString(cudaGetLastError()));
      break;
    }
    b->nprim_sig_h.resize(np);
    for (int k = 0; k < np; ++k) b->nprim_sig_h[k] = info_h[k].nprim;
    // Ket lists: the pairs of each class in buckets of equal significant
    // primitive-pair count (descending), Q descending inside a bucket, so
    // the 32 lanes of a warp loop over the same number of primitives and
    // the Schwarz-surviving kets of a bucket are a prefix of it.
    b->ketlist_h.resize(np);
    for (int X = 0; X < HF_NPAIRCLASS; ++X) {
      const int s0 = b->class_begin[X], s1 = b->class_begin[X + 1];
      for (int k = s0; k < s1; ++k) b->ketlist_h[k] = k;
      std::stable_sort(b->ketlist_h.begin() + s0, b->ketlist_h.begin() + s1, [&](int x, int y) {
        if (b->nprim_sig_h[x] != b->nprim_sig_h[y]) return b->nprim_sig_h[x] > b->nprim_sig_h[y];
        return b->Q_h[x] > b->Q_h[y];
      });
      b->buckets[X].clear();
      for (int k = s0; k < s1; ++k)
        if (k == s0 || b->nprim_sig_h[b->ketlist_h[k]] != b->nprim_sig_h[b->ketlist_h[k - 1]])
          b->buckets[X].push_back(k - s0);
      b->buckets[X].push_back(s1 - s0);
    }
    if (cudaMemcpyAsync(b->ketlist.ptr, b->ketlist_h.data(), sizeof(int) * np, cudaMemcpyHostToDevice, st) !=
        cudaSuccess) {
      rc = hf_fail(HF_ERR_CUDA, "upload");
      break;
    }
  } while (0);
  if (rc != HF_OK) {
    cudaStreamSynchronize(st);
    hf_basis_destroy(b);
    return rc;
  }
  *out = b;
  return HF_OK;
}

extern "C" void hf_basis_destroy(hf_basis* b) {
  if (!b) return;
  hf_ctx* ctx = b->ctx;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  delete b;
  // the last basis of a context whose destroy was called finishes it
  if (ctx->live_bases.fetch_sub(1) == 1 && ctx->destroy_pending.load()) hf_ctx_teardown(ctx);
}

extern "C" int hf_basis_nbf(const hf_basis* b) { return b ? b->nbf : 0; }
extern "C" int hf_basis_nshell(const hf_basis* b) { return b ? b->nshell : 0; }

extern "C" size_t hf_basis_device_bytes(const hf_basis* b) {
  if (!b) return 0;
  size_t s = b->prim64.bytes() + b->prim32.bytes() + b->primdf.bytes() + b->pinfo.bytes() + b->Q.bytes() + b->ketlist.bytes() +
             b->counters.bytes() + b->hD.bytes() + b->hJ.bytes() + b->hK.bytes() + b->Dsum.bytes() + b->detq.bytes() + b->S.bytes() + b->T.bytes() +
             b->V.bytes();
  for (int c = 0; c < HF_NCLASS; ++c)
    for (const ClassWork* w : {&b->work64[c], &b->work32[c]})
      s += w->bra.bytes() + w->kbeg.bytes() + w->kend.bytes() + w->ioff.bytes() + w->nsplit.bytes();
  return s;
}

// ------------------------------------------------------------- Schwarz output
extern "C" int hf_schwarz(hf_basis* b, double* Q) {
  if (!b || !Q) return hf_fail(HF_ERR_INVALID, "hf_schwarz: null argument");
  const int ns = b->nshell;
  for (int k = 0; k < ns * ns; ++k) Q[k] = 0.0;
  for (int k = 0; k < b->npairs; ++k) {
    const int A = b->pair_A[k], B = b->pair_B[k];
    Q[A * ns + B] = Q[B * ns + A] = b->Q_h[k];
  }
  return HF_OK;
}

// ------------------------------------------------------------- work lists
// For each canonical class (X|Y), X >= Y: every pair of class X is a bra;
// its kets are taken bucket by bucket from the class-Y list.  Inside a
// bucket (Q descending) the kept kets are the prefix with Q_i Q_k >= tau
// (the Schwarz rule: drop iff Q_ab Q_cd < tau); when X == Y only kets at
// list positions <= the bra's own position are taken, so each unordered
// pair of pairs appears once.  Kets with Q_i Q_k >= fp32_bound form the
// FP64 range of the entry, the rest its FP32 range.
int hf_basis_prepare_work(hf_basis* b, double tau, double fp32_bound, unsigned flags) {
  const bool rys = (flags & HF_JK_RYS) != 0;
  if (b->have_work && b->work_tau == tau && b->work_fp32 == fp32_bound && b->work_rys == rys) return HF_OK;
  hf_ctx* ctx = b->ctx;
  cudaStream_t st = ctx->stream;
  for (int X = 0; X < HF_NPAIRCLASS; ++X)
    for (int Y = 0; Y <= X; ++Y) {
      const int cls = X * (X + 1) / 2 + Y;
      const int xb = b->class_begin[X], xe = b->class_begin[X + 1];
      const int yb = b->class_begin[Y];
      const std::vector<int>& bk = b->buckets[Y];
      // Rys lists (f/g classes, or every class under HF_JK_RYS): one ket
      // per item, each item split into the class's output chunks
      const bool rys_list = rys || (ctx->ops[cls].rys_native && ctx->ops[cls].chunk == 1);
      const int chunk = rys_list ? 1 : ctx->ops[cls].chunk;
      const int nchunk = rys_list ? ctx->ops[cls].rys_nchunks : 0;
      std::vector<int> bra[2], kb[2], ke[2], io[2], sp[2];
      long long nq[2] = {0, 0};
      io[0].push_back(0);
      io[1].push_back(0);
      for (int i = xb; i < xe; ++i) {
        const int pi = b->ketlist_h[i];
        const double qi = b->Q_h[pi];
        const int ipos = i - xb;  // the bra's position in the class-X list (== class-Y list when X == Y)
        for (size_t u = 0; u + 1 < bk.size(); ++u) {
          const int b0 = bk[u], b1 = bk[u + 1];
          if (X == Y && b0 > ipos) break;
          auto count_ge = [&](double thr) {  // first position in [b0, b1) with qi * Q < thr
            int lo = b0, hi = b1;
            while (lo < hi) {
              const int mid = (lo + hi) / 2;
              if (qi * b->Q_h[b->ketlist_h[yb + mid]] >= thr) lo = mid + 1; else hi = mid;
            }
            return lo;
          };
          int n = count_ge(tau);
          if (X == Y) n = std::min(n, ipos + 1);
          const int m = fp32_bound > 0.0 ? std::min(count_ge(fp32_bound), n) : n;
          const int lo_[2] = {b0, m}, hi_[2] = {m, n};
          for (int r = 0; r < 2; ++r) {
            const int cnt = hi_[r] - lo_[r];
            if (cnt <= 0) continue;
            bra[r].push_back(pi);
            kb[r].push_back(lo_[r]);
            ke[r].push_back(hi_[r]);
            nq[r] += cnt;
          }
        }
      }
      // Item split along the primitive loop.  A class whose work is small
      // next to the GPU is bound by its longest items (a lane walks up to
      // nb x nk primitive quartets in series), so when the class's work per
      // resident warp is below an item's length, the long items are cut
      // into parts of about that length: bra primitive pairs for the
      // thread-per-quartet kernels, primitive quartets (whole rounds of 32)
      // for the warp-cooperative ones, any primitive-quartet range for the
      // Rys kernel (whose items are further multiplied by its output
      // chunks).  Large workloads are not split.
      const int yb_ = b->class_begin[Y];
      for (int r = 0; r < 2; ++r) {
        const size_t ne = bra[r].size();
        std::vector<long long> len(ne);
        long long work = 0;
        for (size_t e = 0; e < ne; ++e) {
          const long long nbp = b->nprim_sig_h[bra[r][e]];
          const long long nkp = b->nprim_sig_h[b->ketlist_h[yb_ + kb[r][e]]];  // uniform inside a bucket
          len[e] = nbp * nkp;  // primitive quartets per lane (per warp for the cooperative kernels)
          work += len[e] * ((ke[r][e] - kb[r][e] + chunk - 1) / chunk) * std::max(1, nchunk);
        }
        const long long warps = 16LL * ctx->num_sms;
        const long long floor_len = rys_list ? 16 : chunk == 1 ? 64 : 16;
        const long long target = std::max(floor_len, work / std::max(1LL, warps));
        sp[r].resize(ne);
        for (size_t e = 0; e < ne; ++e) {
          const long long nbp = b->nprim_sig_h[bra[r][e]];
          long long parts = (len[e] + target - 1) / target;
          parts = std::min(parts, rys_list ? std::max(1LL, len[e])
                                           : chunk == 1 ? std::max(1LL, (len[e] + 31) / 32) : std::max(1LL, nbp));
          parts = std::max(1LL, parts);
          if (rys_list) parts = std::min(parts * nchunk, (long long)(1 << 20)) / nchunk * nchunk;
          sp[r][e] = (int)parts;
          // item offsets are int on the device: checked in 64 bits, per entry
          const long long next =
              (long long)io[r].back() + (long long)((ke[r][e] - kb[r][e] + chunk - 1) / chunk) * sp[r][e];
          if (next > (1 << 30)) return hf_fail(HF_ERR_TOO_LARGE, "class %d: too many work items", cls);
          io[r].push_back((int)next);
        }
      }
      for (int r = 0; r < 2; ++r) {
        ClassWork& w = r == 0 ? b->work64[cls] : b->work32[cls];
        const int nb = (int)bra[r].size();
        HF_CHECK(w.bra.alloc(ctx, nb));
        HF_CHECK(w.kbeg.alloc(ctx, nb));
        HF_CHECK(w.kend.alloc(ctx, nb));
        HF_CHECK(w.ioff.alloc(ctx, nb + 1));
        HF_CHECK(w.nsplit.alloc(ctx, nb));
        if (nb > 0) {
          HF_CUDA(cudaMemcpyAsync(w.bra.ptr, bra[r].data(), sizeof(int) * nb, cudaMemcpyHostToDevice, st));
          HF_CUDA(cudaMemcpyAsync(w.kbeg.ptr, kb[r].data(), sizeof(int) * nb, cudaMemcpyHostToDevice, st));
          HF_CUDA(cudaMemcpyAsync(w.kend.ptr, ke[r].data(), sizeof(int) * nb, cudaMemcpyHostToDevice, st));
          HF_CUDA(cudaMemcpyAsync(w.ioff.ptr, io[r].data(), sizeof(int) * (nb + 1), cudaMemcpyHostToDevice, st));
          HF_CUDA(cudaMemcpyAsync(w.nsplit.ptr, sp[r].data(), sizeof(int) * nb, cudaMemcpyHostToDevice, st));
        }
        w.w.bra = w.bra.ptr;
        w.w.ket = b->ketlist.ptr + yb;
        w.w.kbeg = w.kbeg.ptr;
        w.w.kend = w.kend.ptr;
        w.w.ioff = w.ioff.ptr;
        w.w.mol = nullptr;
        w.w.nsplit = w.nsplit.ptr;
        w.w.nbra = nb;
        w.w.nitems = io[r].back();
        w.w.counter = b->counters.ptr + 2 * cls + r;
        w.w.chunk = chunk;
        w.w.nchunk = nchunk;
        w.nquartets = nq[r];
        w.bra_h = std::move(bra[r]);
        w.kbeg_h = std::move(kb[r]);
        w.kend_h = std::move(ke[r]);
        w.nsplit_h = std::move(sp[r]);
      }
    }
  // the host vectors above are consumed by the async copies: wait for them
  HF_CUDA(cudaStreamSynchronize(st));
  b->have_work = true;
  b->work_tau = tau;
  b->work_fp32 = fp32_bound;
  b->work_rys = rys;
  return HF_OK;
}

extern "C" int hf_count_quartets(hf_basis* b, const hf_jk_opts* opts, long long* n_total, long long* n_fp32) {
  if (!b) return hf_fail(HF_ERR_INVALID, "null basis");
  hf_jk_opts o;
  hf_jk_opts_default(&o);
  if (opts) o = *opts;
  std::lock_guard<std::mutex> lk(b->ctx->mu);
  cudaSetDevice(b->ctx->device);
  HF_CHECK(hf_basis_prepare_work(b, o.schwarz_tau, o.fp32_bound, o.flags));
  long long t = 0, f = 0;
  for (int c = 0; c < HF_NCLASS; ++c) {
    t += b->work64[c].nquartets + b->work32[c].nquartets;
    f += b->work32[c].nquartets;
  }
  if (n_total) *n_total = t;
  if (n_fp32) *n_fp32 = f;
  return HF_OK;
}

int hf_launch_grid(hf_ctx* ctx, int occ, int nitems) {
  const int warps = 4;
  int g = (nitems + warps - 1) / warps;
  const int cap = std::max(1, occ) * ctx->num_sms;
  return std::max(1, std::min(g, cap));
}

LaunchShape hf_launch_shape(const hf_ctx* ctx, int occ, int nitems, int cap_per_sm) {
  const int per_sm = std::max(1, cap_per_sm > 0 ? std::min(occ, cap_per_sm) : occ);
  const int g = (int)std::min<long long>((nitems + 3LL) / 4, (long long)per_sm * ctx->num_sms);
  return LaunchShape{std::max(1, g), 128};
}

int hf_jk_run(hf_basis* b, const double* D, double* Jp, double* Kp, double* J, double* K, int* counters,
              const hf_jk_opts& o, cudaStream_t st, long long* nq, JKClassTiming* timing, const JKSpin* spin) {
  NvtxRange nv_build("J/K build");
  hf_ctx* ctx = b->ctx;
  const PairSet ps = hf_pairset(b);
  KernelCommon kc = hf_kernel_common(ctx, o.flags);
  const size_t nn = (size_t)b->nbf * b->nbf;
  MolJK one{D, Jp, Kp, b->nbf, 0};
  if (spin) {
    one.Dj = spin->Dj;
    one.D2 = spin->D2;
    one.K2 = spin->K2;
  }
  // deterministic order: the kernels accumulate into fixed-point words
  // (basis-owned, zeroed here) and finish_fixed writes J, K (and K2)
  const bool det = (o.flags & HF_JK_DETERMINISTIC) != 0;
  unsigned long long* q = nullptr;
  if (det) {
    const size_t words = 2 * nn * (spin ? 3 : 2);
    if (b->detq.n < words) HF_CHECK(b->detq.alloc(ctx, words));
    q = b->detq.ptr;
    HF_CUDA(cudaMemsetAsync(q, 0, words * sizeof(unsigned long long), st));
    kc.det = 1;
    one.J = reinterpret_cast<double*>(q);
    one.K = reinterpret_cast<double*>(q + 2 * nn);
    if (spin) one.K2 = reinterpret_cast<double*>(q + 4 * nn);
  }
  long long total = 0;
  if (timing) {
    timing->n = 0;
    HF_CUDA(cudaEventRecord(timing->ev[timing->n++], st));
  }
  // heaviest classes first.  The f/g (Rys) classes are many and often
  // small: without per-class timing they fork onto the side streams (round
  // robin) and run beside each other and the s/p/d classes; every class
  // shares only the J/K atomics with the others.
  bool forked = false;
  int nside = 0;
  for (int c = HF_NCLASS - 1; c >= 0; --c) {
    const EriClassOps& op = ctx->ops[c];
    for (int r = 0; r < 2; ++r) {
      const ClassWork& cw = r == 0 ? b->work64[c] : b->work32[c];
      total += cw.nquartets;
      if (cw.w.nitems <= 0) continue;
      JKWork w = cw.w;
      w.counter = counters + 2 * c + r;
      const jk_launch_fn fn = r == 0 ? hf_jk_hi(op, o.flags) : hf_jk_lo(op, o.flags);
      const int occ = r == 0 ? hf_occ_hi(op, o.flags) : hf_occ_lo(op, o.flags);
      const LaunchShape sh = hf_launch_shape(ctx, occ, w.nitems);
      NvtxRange nv_cls(op.name);
      cudaStream_t ls = st;
      if (!timing && (op.rys_native || (o.flags & HF_JK_RYS))) {
        if (!forked) {
          HF_CUDA(cudaEventRecord(ctx->fork_ev, st));
          for (int k = 0; k < hf_ctx::kSide; ++k) HF_CUDA(cudaStreamWaitEvent(ctx->side[k], ctx->fork_ev, 0));
          forked = true;
        }
        ls = ctx->side[nside++ % hf_ctx::kSide];
      }
      fn(w, ps, kc, one, nullptr, sh.grid, sh.threads, ls);
      if (timing) {
        timing->which[timing->n - 1] = 2 * c + r;
        HF_CUDA(cudaEventRecord(timing->ev[timing->n++], st));
      }
    }
  }
  HF_CUDA(cudaGetLastError());
  if (forked)
    for (int k = 0; k < hf_ctx::kSide; ++k) {
      HF_CUDA(cudaEventRecord(ctx->join_ev[k], ctx->side[k]));
      HF_CUDA(cudaStreamWaitEvent(st, ctx->join_ev[k], 0));
    }
  double* K2 = spin ? spin->K2 : nullptr;
  if (det)
    finish_fixed<<<(unsigned)((nn + 255) / 256), 256, 0, st>>>(q, q + 2 * nn, spin ? q + 4 * nn : nullptr, J, K, K2,
                                                               b->nbf);
  else
    symmetrize_jk<<<(unsigned)((nn + 255) / 256), 256, 0, st>>>(Jp, Kp, J, K, K2, K2, b->nbf);
  HF_CUDA(cudaGetLastError());
  HF_CHECK(hf_bounds_status(ctx, "J/K build"));
  if (nq) *nq = total;
  return HF_OK;
}

int hf_fock_jk_device(hf_basis* b, const double* D, double* J, double* K, const hf_jk_opts& o, long long* nq) {
  hf_ctx* ctx = b->ctx;
  cudaStream_t st = ctx->stream;
  HF_CHECK(hf_basis_prepare_work(b, o.schwarz_tau, o.fp32_bound, o.flags));
  const size_t nn = (size_t)b->nbf * b->nbf;
  HF_CUDA(cudaMemsetAsync(J, 0, nn * sizeof(double), st));
  HF_CUDA(cudaMemsetAsync(K, 0, nn * sizeof(double), st));
  HF_CUDA(cudaMemsetAsync(b->counters.ptr, 0, sizeof(int) * 2 * HF_NCLASS, st));
  return hf_jk_run(b, D, J, K, J, K, b->counters.ptr, o, st, nq, nullptr);
}

// Operations per primitive quartet outside the VRR: p+q, 1/sqrt, 1/(p+q),
// rho/p, rho/q, PQ, WP, WQ, T, prefactor (22), the Boys evaluation (index
// 3, Horner 14 per order for L <= 1; else 3 + 14 + exp 14 + 3L), scaling
// of B (L+1).
static int prim_overhead_flops(int L) {
  const int boys = L <= 1 ? 3 + 14 * (L + 1) : 3 + 14 + 14 + 3 * L;
  return 22 + boys + (L + 1);
}

extern "C" int hf_class_stats_get(hf_basis* b, const hf_jk_opts* opts, hf_class_stats* out) {
  if (!b || !out) return hf_fail(HF_ERR_INVALID, "hf_class_stats_get: null argument");
  hf_jk_opts o;
  hf_jk_opts_default(&o);
  if (opts) o = *opts;
  std::lock_guard<std::mutex> lk(b->ctx->mu);
  cudaSetDevice(b->ctx->device);
  HF_CHECK(hf_basis_prepare_work(b, o.schwarz_tau, o.fp32_bound, o.flags));
  // prefix sums of significant primitive-pair counts along each class's ket list
  std::vector<long long> pre(b->npairs + 1, 0);
  for (int k = 0; k < b->npairs; ++k) pre[k + 1] = pre[k] + b->nprim_sig_h[b->ketlist_h[k]];
  for (int X = 0; X < HF_NPAIRCLASS; ++X)
    for (int Y = 0; Y <= X; ++Y) {
      const int c = X * (X + 1) / 2 + Y;
      hf_class_stats& st = out[c];
      pair_ls(X, &st.la, &st.lb);
      pair_ls(Y, &st.lc, &st.ld);
      const EriClassOps& op = b->ctx->ops[c];
      const int L = st.la + st.lb + st.lc + st.ld;
      st.vrr_flops = op.vrr_flops;
      st.hrr_flops = op.hrr_flops;
      // the Rys classes' count already holds their set-up and quadrature rule
      st.prim_flops = op.vrr_flops + (op.jk64 == op.jkrys ? 0 : prim_overhead_flops(L));
      const int nblk = ((st.la + 1) * (st.la + 2) / 2) * ((st.lb + 1) * (st.lb + 2) / 2) *
                       ((st.lc + 1) * (st.lc + 2) / 2) * ((st.ld + 1) * (st.ld + 2) / 2);
      st.digest_flops = 6 * 2 * nblk;
      const int yb = b->class_begin[Y];
      for (int r = 0; r < 2; ++r) {
        ClassWork& w = r == 0 ? b->work64[c] : b->work32[c];
        const std::vector<int>& bra = w.bra_h;
        const std::vector<int>& kb = w.kbeg_h;
        const std::vector<int>& ke = w.kend_h;
        long long pq = 0;
        for (int i = 0; i < w.w.nbra; ++i)
          pq += (long long)b->nprim_sig_h[bra[i]] * (pre[yb + ke[i]] - pre[yb + kb[i]]);
        if (r == 0) { st.quartets_fp64 = w.nquartets; st.prim_quartets_fp64 = pq; }
        else { st.quartets_fp32 = w.nquartets; st.prim_quartets_fp32 = pq; }
      }
    }
  return HF_OK;
}

extern "C" int hf_fock_jk_profiled(hf_basis* b, const double* D, double* J, double* K, const hf_jk_opts* opts,
                                   double* class_ms) {
  if (!b || !D || !J || !K || !class_ms) return hf_fail(HF_ERR_INVALID, "hf_fock_jk_profiled: null argument");
  hf_jk_opts o;
  hf_jk_opts_default(&o);
  if (opts) o = *opts;
  if (!(o.schwarz_tau >= 0.0) || !(o.fp32_bound >= 0.0)) return hf_fail(HF_ERR_INVALID, "negative threshold");
  hf_ctx* ctx = b->ctx;
  std::lock_guard<std::mutex> lk(ctx->mu);
  cudaSetDevice(ctx->device);
  cudaStream_t st = ctx->stream;
  HF_CHECK(hf_basis_prepare_work(b, o.schwarz_tau, o.fp32_bound, o.flags));
  const size_t nn = (size_t)b->nbf * b->nbf;
  HF_CUDA(cudaMemsetAsync(J, 0, nn * sizeof(double), st));
  HF_CUDA(cudaMemsetAsync(K, 0, nn * sizeof(double), st));
  HF_CUDA(cudaMemsetAsync(b->counters.ptr, 0, sizeof(int) * 2 * HF_NCLASS, st));
  JKClassTiming tm;
  for (auto& e : tm.ev) HF_CUDA(cudaEventCreate(&e));
  const int rc = hf_jk_run(b, D, J, K, J, K, b->counters.ptr, o, st, nullptr, &tm);
  if (rc == HF_OK) {
    HF_CUDA(cudaStreamSynchronize(st));
    for (int k = 0; k < 2 * HF_NCLASS; ++k) class_ms[k] = 0.0;
    for (int k = 0; k + 1 < tm.n; ++k) {
      float ms = 0.f;
      HF_CUDA(cudaEventElapsedTime(&ms, tm.ev[k], tm.ev[k + 1]));
      class_ms[tm.which[k]] = ms;
    }
  }
  for (auto& e : tm.ev) cudaEventDestroy(e);
  return rc;
}

extern "C" int hf_fock_jk(hf_basis* b, const double* D, double* J, double* K, const hf_jk_opts* opts) {
  if (!b || !D || !J || !K) return hf_fail(HF_ERR_INVALID, "hf_fock_jk: null argument");
  hf_jk_opts o;
  hf_jk_opts_default(&o);
  if (opts) o = *opts;
  if (!(o.schwarz_tau >= 0.0) || !(o.fp32_bound >= 0.0)) return hf_fail(HF_ERR_INVALID, "negative threshold");
  hf_ctx* ctx = b->ctx;
  std::lock_guard<std::mutex> lk(ctx->mu);
  cudaSetDevice(ctx->device);
  cudaStream_t st = ctx->stream;
  const size_t nn = (size_t)b->nbf * b->nbf;
  if (o.flags & HF_JK_HOST) {
    if (b->hD.n != nn) {
      HF_CHECK(b->hD.alloc(ctx, nn));
      HF_CHECK(b->hJ.alloc(ctx, nn));
      HF_CHECK(b->hK.alloc(ctx, nn));
    }
    HF_CUDA(cudaMemcpyAsync(b->hD.ptr, D, nn * sizeof(double), cudaMemcpyHostToDevice, st));
    HF_CHECK(hf_fock_jk_device(b, b->hD.ptr, b->hJ.ptr, b->hK.ptr, o, nullptr));
    HF_CUDA(cudaMemcpyAsync(J, b->hJ.ptr, nn * sizeof(double), cudaMemcpyDeviceToHost, st));
    HF_CUDA(cudaMemcpyAsync(K, b->hK.ptr, nn * sizeof(double), cudaMemcpyDeviceToHost, st));
  } else {
    HF_CHECK(hf_fock_jk_device(b, D, J, K, o, nullptr));
  }
  HF_CUDA(cudaStreamSynchronize(st));
  return HF_OK;
}

__global__ void add_densities(const double* __restrict__ A, const double* __restrict__ B, double* __restrict__ C,
                              size_t nn) {
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t < nn) C[t] = A[t] + B[t];
}

int hf_fock_jk_uhf_device(hf_basis* b, const double* Da, const double* Db, const double* Dsum, double* J, double* Ka,
                          double* Kb, const hf_jk_opts& o, long long* nq) {
  hf_ctx* ctx = b->ctx;
  cudaStream_t st = ctx->stream;
  HF_CHECK(hf_basis_prepare_work(b, o.schwarz_tau, o.fp32_bound, o.flags));
  const size_t nn = (size_t)b->nbf * b->nbf;
  HF_CUDA(cudaMemsetAsync(J, 0, nn * sizeof(double), st));
  HF_CUDA(cudaMemsetAsync(Ka, 0, nn * sizeof(double), st));
  HF_CUDA(cudaMemsetAsync(Kb, 0, nn * sizeof(double), st));
  HF_CUDA(cudaMemsetAsync(b->counters.ptr, 0, sizeof(int) * 2 * HF_NCLASS, st));
  const JKSpin spin{Dsum, Db, Kb};
  return hf_jk_run(b, Da, J, Ka, J, Ka, b->counters.ptr, o, st, nq, nullptr, &spin);
}

extern "C" int hf_fock_jk_uhf(hf_basis* b, const double* Da, const double* Db, double* J, double* Ka, double* Kb,
                              const hf_jk_opts* opts) {
  if (!b || !Da || !Db || !J || !Ka || !Kb) return hf_fail(HF_ERR_INVALID, "hf_fock_jk_uhf: null argument");
  hf_jk_opts o;
  hf_jk_opts_default(&o);
  if (opts) o = *opts;
  if (!(o.schwarz_tau >= 0.0) || !(o.fp32_bound >= 0.0)) return hf_fail(HF_ERR_INVALID, "negative threshold");
  if (o.flags & HF_JK_HOST) return hf_fail(HF_ERR_INVALID, "hf_fock_jk_uhf: device pointers only");
  hf_ctx* ctx = b->ctx;
  std::lock_guard<std::mutex> lk(ctx->mu);
  cudaSetDevice(ctx->device);
  cudaStream_t st = ctx->stream;
  const size_t nn = (size_t)b->nbf * b->nbf;
  if (b->Dsum.n != nn) HF_CHECK(b->Dsum.alloc(ctx, nn));
  add_densities<<<(unsigned)((nn + 255) / 256), 256, 0, st>>>(Da, Db, b->Dsum.ptr, nn);
  HF_CUDA(cudaGetLastError());
  HF_CHECK(hf_fock_jk_uhf_device(b, Da, Db, b->Dsum.ptr, J, Ka, Kb, o, nullptr));
  HF_CUDA(cudaStreamSynchronize(st));
  return HF_OK;
}

// ------------------------------------------------------------- ERI tensor
extern "C" int hf_eri_tensor(hf_basis* b, double* G) {
  if (!b || !G) return hf_fail(HF_ERR_INVALID, "hf_eri_tensor: null argument");
  if (b->nbf > HF_STORED_NBF_MAX)
    return hf_fail(HF_ERR_INVALID, "hf_eri_tensor: nbf %d above %d", b->nbf, HF_STORED_NBF_MAX);
  hf_ctx* ctx = b->ctx;
  std::lock_guard<std::mutex> lk(ctx->mu);
  cudaSetDevice(ctx->device);
  HF_CHECK(hf_eri_tensor_device(b, G));
  HF_CUDA(cudaStreamSynchronize(ctx->stream));
  return HF_OK;
}

int hf_eri_tensor_device(hf_basis* b, double* G) {
  hf_ctx* ctx = b->ctx;
  cudaStream_t st = ctx->stream;
  HF_CHECK(hf_basis_prepare_work(b, 0.0, 0.0, 0u));
  HF_CUDA(cudaMemsetAsync(b->counters.ptr, 0, sizeof(int) * 2 * HF_NCLASS, st));
  const PairSet ps = hf_pairset(b);
  const KernelCommon kc = hf_kernel_common(ctx, 0);
  for (int c = 0; c < HF_NCLASS; ++c) {
    ClassWork& w = b->work64[c];
    if (w.w.nitems > 0) ctx->ops[c].store(w.w, ps, kc, G, b->nbf, hf_launch_grid(ctx, 4, w.w.nitems), st);
  }
  HF_CUDA(cudaGetLastError());
  return HF_OK;
}

// J_ij = sum_kl G_ijkl D_kl and K_il = sum_jk G_ijkl D_jk: one warp per output
// element.  The tensor holds every permutation image of Eq. 5, so the K sum
// reads (ip|xq) = (ip|qx): consecutive lanes take consecutive q in both sums,
// and each warp reads n^2 contiguous doubles.
__global__ void jk_stored_kernel(const double* __restrict__ G, const double* __restrict__ D, double* __restrict__ J,
                                 double* __restrict__ K, int n) {
  const long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const long long nn = (long long)n * n;
  if (w >= 2 * nn) return;
  const bool isK = w >= nn;
  const long long e = isK ? w - nn : w;
  const int i = (int)(e / n), x = (int)(e % n);
  double s = 0.0;
  for (long long t = lane; t < nn; t += 32) {
    const int p = (int)(t / n), q = (int)(t % n);
    if (!isK) s += G[(((size_t)i * n + x) * n + p) * n + q] * D[(size_t)p * n + q];       // J_ix, (ix|pq) D_pq
    else s += G[(((size_t)i * n + p) * n + x) * n + q] * D[(size_t)p * n + q];           // K_ix, (ip|xq) D_pq
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) (isK ? K : J)[(size_t)i * n + x] = s;
}

int hf_jk_stored_device(hf_basis* b, const double* G, const double* D, double* J, double* K) {
  const long long threads = 2LL * b->nbf * b->nbf * 32;
  jk_stored_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, b->ctx->stream>>>(G, D, J, K, b->nbf);
  HF_CUDA(cudaGetLastError());
  return HF_OK;
}

extern "C" int hf_jk_stored(hf_basis* b, const double* G, const double* D, double* J, double* K) {
  if (!b || !G || !D || !J || !K) return hf_fail(HF_ERR_INVALID, "hf_jk_stored: null argument");
  if (b->nbf > HF_STORED_NBF_MAX)
    return hf_fail(HF_ERR_INVALID, "hf_jk_stored: nbf %d above %d", b->nbf, HF_STORED_NBF_MAX);
  hf_ctx* ctx = b->ctx;
  std::lock_guard<std::mutex> lk(ctx->mu);
  cudaSetDevice(ctx->device);
  HF_CHECK(hf_jk_stored_device(b, G, D, J, K));
  HF_CUDA(cudaStreamSynchronize(ctx->stream));
  return HF_OK;
}
