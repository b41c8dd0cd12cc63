// multi.h -- one launch per angular class over the quartets of many molecules.
#pragma once
#include <vector>

#include "hf_internal.h"

// A set of molecules whose J/K builds run together: for every (class,
// precision) the molecules' work entries are concatenated, each tagged with
// its molecule, and one persistent kernel per class covers them all.  Each
// molecule keeps its own pair data, ket lists and D/J/K buffers (MolJK).
struct MultiJK {
  hf_ctx* ctx = nullptr;
  int nmol = 0;
  std::vector<MolJK> table_h;
  DevArray<MolJK> table;
  DevArray<int> bra[2 * HF_NCLASS], kbeg[2 * HF_NCLASS], kend[2 * HF_NCLASS], ioff[2 * HF_NCLASS],
      mol[2 * HF_NCLASS], nsplit[2 * HF_NCLASS];
  JKWork w[2 * HF_NCLASS] = {};
  long long nquartets[2 * HF_NCLASS] = {};
  std::vector<long long> mol_quartets;  // per molecule, all classes
  DevArray<int> counters;
  int grid_scale[HF_NCLASS] = {};       // blocks per SM per class chosen by the tuner (0 = full occupancy)
  unsigned jk_flags = 0;                // HF_JK_* of the launches (precision tiers)

  // mols[i] with density/outputs D[i], J[i], K[i]; every basis must have its
  // work lists prepared for the same options.  Rebuilds all device lists.
  int build(hf_ctx* c, const std::vector<hf_basis*>& mols, const std::vector<const double*>& D,
            const std::vector<double*>& J, const std::vector<double*>& K);
  // Mark molecules active/inactive (uploads the table).
  int set_active(const std::vector<int>& active);
  // Make molecule m's build unrestricted: J from Dj (D^a + D^b), K from its
  // D (alpha) and K2 from D2 (beta) in the same launch (uploads the table).
  int set_spin(int m, const double* Dj, const double* D2, double* K2);
  // Zero J/K of active molecules, run all classes, symmetrise.  With
  // class_ms, each class launch is bracketed by events and its duration in
  // ms is added to class_ms[cls] (the caller synchronises).
  int launch(const KernelCommon& kc, double* class_ms = nullptr);
  // Autotuner, online: each call runs one J/K build of the current set with
  // the next candidate blocks-per-SM setting (full occupancy, 2, 1), timing
  // every class with events; after the last candidate each class keeps its
  // fastest setting.  The builds are the SCF's own iterations (same quartet
  // work each time), so tuning costs no extra builds.
  int tune_step(const KernelCommon& kc);
  bool tuned = false;
  int tune_iter = 0;
  double tune_ms[3][HF_NCLASS] = {};
  // Capture launch() into a CUDA graph (replayed by run()); the graph stays
  // valid across set_active() since only the table's contents change.
  int capture(const KernelCommon& kc);
  int run(const KernelCommon& kc);
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  bool capturing = false;  // inside capture(): no host reads of device status
  ~MultiJK();
};
