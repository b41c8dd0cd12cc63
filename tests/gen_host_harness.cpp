// Host build of the generated per-class recurrence code (test
// infrastructure): the straight-line VRR and HRR bodies of
// paper_1303_4916_gb300/csrc/eri_classes.cuh, compiled for the CPU with the
// device qualifiers defined away, behind plain C entry points that
// tests/test_codegen_host.py calls through ctypes.
#include <cmath>
#define __device__
#define __forceinline__ inline
using std::fma;
using std::fmaf;
#include "eri_classes.cuh"

// q = PA[3] WP[3] QC[3] WQ[3] o2p o2q o2pq rp rq
#define HF_HOST_WRAP(NAME, la, lb, lc, ld, vf, hf)                                                   \
  extern "C" void vrr_##NAME(double* acc, const double* B, const double* q) {                      \
    for (int x = 0; x < hfgen::NAME::NE * hfgen::NAME::NF; ++x) acc[x] = 0.0;                       \
    hfgen::NAME::vrr<double>(acc, B, q, q + 3, q + 6, q + 9, q[12], q[13], q[14], q[15], q[16]);    \
  }                                                                                                  \
  extern "C" void hrr_##NAME(const double* acc, double* out, const double* AB, const double* CD) {  \
    hfgen::NAME::hrr<double>(acc, out, AB, CD);                                                      \
  }
HF_GEN_CLASS_TABLE(HF_HOST_WRAP)
