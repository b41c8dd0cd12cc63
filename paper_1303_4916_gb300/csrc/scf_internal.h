// scf_internal.h -- per-molecule SCF state (device buffers + DIIS bookkeeping).
#pragma once
#include <vector>

#include "hf_internal.h"

struct ScfState {
  int n = 0, m = 0;
  DevArray<double> H, X, F, Fk, W, C, D, J, K, T1, T2, eps, scal, work, Fring, Ering, F1;
  DevArray<int> islots, info;
  int lwork = 0;
  double smin = 0.0;
  // iteration state
  int iter = 0, converged = 0;
  double energy = 0.0, e_old = 0.0, delta_e = 0.0, diis_error = 0.0;
  std::vector<int> slots;  // DIIS ring slots in use, oldest first
  int next = 0;
  double Bslot[16 * 16] = {};
  long long fock_builds = 0, quartets = 0;
  bool have_F1 = false;
  double* hscal = nullptr;   // pinned: scalars from the device (energy, |e|max, DIIS dots)
  double* hcoef = nullptr;   // pinned: DIIS coefficients to the device
  int* hslots = nullptr;     // pinned: DIIS slot order to the device
  ScfState() = default;
  ScfState(const ScfState&) = delete;
  ScfState& operator=(const ScfState&) = delete;
  ~ScfState() {
    if (hscal) cudaFreeHost(hscal);
  }
};

int scf_state_init(hf_basis* b, ScfState& s, int diis_size);
int scf_setup(hf_basis* b, ScfState& s);
int scf_begin(hf_basis* b, ScfState& s, const hf_scf_opts& o, const double* G);
int scf_iterate(hf_basis* b, ScfState& s, const hf_scf_opts& o, const double* G);
int scf_density(hf_basis* b, ScfState& s);
int scf_post_jk(hf_basis* b, ScfState& s);
int scf_diis_step(hf_basis* b, ScfState& s);
bool scf_after_iter(hf_basis* b, ScfState& s, const hf_scf_opts& o);
int scf_finish(hf_basis* b, ScfState& s, hf_scf_result* r);
