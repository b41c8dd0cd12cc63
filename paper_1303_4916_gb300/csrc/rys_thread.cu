// rys_thread.cu -- the small f/g classes (at most 30 outputs per quartet:
// (fs|ss), (fp|ss), (fs|ps), (gs|ss)) by Rys quadrature in the
// thread-per-quartet J/K kernel of eri.cuh, one quartet per lane, so that
// every FP64 instruction of the primitive loop runs on 32 lanes (the
// warp-per-quartet kernel of rys.cu leaves most lanes idle on such small
// blocks).  Own translation unit: the fully unrolled recurrences compile
// beside the other units.
#include <utility>

#include "eri.cuh"
#include "hf_internal.h"

namespace hfr {

constexpr int kThreadOutputs = 30;
template <int LA_, int LB_, int LC_, int LD_>
struct RysT {
  static constexpr int LA = LA_, LB = LB_, LC = LC_, LD = LD_;
  static constexpr int NA = (LA + 1) * (LA + 2) / 2, NB = (LB + 1) * (LB + 2) / 2;
  static constexpr int NC = (LC + 1) * (LC + 2) / 2, ND = (LD + 1) * (LD + 2) / 2;
  static constexpr int NE = 1, NF = 1, L = LA + LB + LC + LD;
  static constexpr bool COOP = false, RYS = true;
};
constexpr int cls_X(int cls) {
  int X = 0;
  while ((X + 1) * (X + 2) / 2 <= cls) ++X;
  return X;
}
constexpr int pc_la(int P) {
  int l = 0;
  while ((l + 1) * (l + 2) / 2 <= P) ++l;
  return l;
}
constexpr int pc_lb(int P) { return P - pc_la(P) * (pc_la(P) + 1) / 2; }
constexpr int cls_Y(int cls) { return cls - cls_X(cls) * (cls_X(cls) + 1) / 2; }
constexpr int ncart_c(int l) { return (l + 1) * (l + 2) / 2; }
constexpr bool thread_class(int cls) {
  const int la = pc_la(cls_X(cls)), lb = pc_lb(cls_X(cls)), lc = pc_la(cls_Y(cls)), ld = pc_lb(cls_Y(cls));
  const int lmax = la > lc ? la : lc;
  return lmax > 2 && ncart_c(la) * ncart_c(lb) * ncart_c(lc) * ncart_c(ld) <= kThreadOutputs;
}
template <int CLS>
using RysTOf = RysT<pc_la(cls_X(CLS)), pc_lb(cls_X(CLS)), pc_la(cls_Y(CLS)), pc_lb(cls_Y(CLS))>;

template <int CLS>
void jk_thread_launch(const JKWork& w, const PairSet& ps, const KernelCommon& kc, const MolJK& one, const MolJK* mols,
                      int grid, int threads, cudaStream_t st) {
  if constexpr (thread_class(CLS)) hfk::eri_jk_kernel<RysTOf<CLS>, double><<<grid, threads, 0, st>>>(w, ps, kc, one, mols);
}
template <int CLS>
int jk_thread_occ() {
  int n = 0;
  if constexpr (thread_class(CLS))
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, hfk::eri_jk_kernel<RysTOf<CLS>, double>, 128, 0);
  return n;
}

template <size_t... I>
void fill(jk_launch_fn* jk, occ_fn* occ, std::index_sequence<I...>) {
  const jk_launch_fn j[] = {(thread_class((int)I) ? &jk_thread_launch<(int)I> : nullptr)...};
  const occ_fn o[] = {(thread_class((int)I) ? &jk_thread_occ<(int)I> : nullptr)...};
  for (int c = 0; c < HF_NCLASS; ++c) {
    jk[c] = j[c];
    occ[c] = o[c];
  }
}

}  // namespace hfr

void hf_rys_thread_classes(jk_launch_fn* jk, occ_fn* occ) {
  hfr::fill(jk, occ, std::make_index_sequence<HF_NCLASS>{});
}
