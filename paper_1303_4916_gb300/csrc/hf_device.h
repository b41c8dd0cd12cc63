// hf_device.h -- data layouts shared by the host runtime and the kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

// Boys tables.  Grid T_i = i * BOYS_H (the double product), i = 0 ..
// BOYS_NGRID-1; lookups use the nearest row, so T < BOYS_TMAX stays inside.
// One slice per order L = 0..BOYS_LMAX; row i of slice L holds the Taylor
// coefficients about T_i of F_L, F_{L+k}(T_i)/k! for k < TERMS (from
// dF_m/dT = -F_{m+1}), followed by those of exp(-T), exp(-T_i)/k!.
// FP64: 8 + 8 coefficients per 128-byte row; FP32: 5 + 5.
#define BOYS_H 0.1
#define BOYS_NGRID 602
#define BOYS_TMAX 60.0
#define BOYS_LMAX 8
#define BOYS_NM 16
#define BOYS64_TERMS 8
#define BOYS64_ROW 16
#define BOYS32_TERMS 5
#define BOYS32_ROW 10
// df64 table: grid T_i = i / 16 (exact in FP32), T < BOYS_TMAX; per row and
// order 16 floats (64 bytes, read as two 256-bit loads): Taylor coefficients
// c_k = F_{L+k}(T_i)/k!, k = 0..4 as (hi, lo) pairs, k = 5..7 as floats, one
// pad, then exp(-T_i) as a (hi, lo) pair.
#define BOYSDF_INV_H 16.0f
#define BOYSDF_NGRID 962
#define BOYSDF_ROW 16
// thread-per-quartet classes with L = la+lb+lc+ld up to this have a df64
// variant; the warp-cooperative classes (L >= 5) take df64 through the
// generic cooperative kernel
#define HF_DF_LMAX 4

// Primitive-pair record, FP64: p, 1/(2p), P[3], PA[3], K, a (80 bytes; a
// is the exponent of A's primitive, b = p - a); FP32: the same ten values
// then two pads (48 bytes); df64: the ten values as (hi, lo) float pairs
// (80 bytes).
// K = c_a c_b exp(-ab/p |AB|^2) sqrt(2) pi^(5/4) / p, so that the
// primitive-quartet prefactor 2 pi^(5/2) / (p q sqrt(p+q)) K_ab K_cd of
// [00|00]^(m) is K_ab' K_cd' / sqrt(p+q).
#define PRIM64_STRIDE 10
#define PRIM32_STRIDE 12
#define PRIMDF_STRIDE 20

// Shell pair (A, B) with l_A >= l_B: first basis functions of A and B,
// offset and count of its significant primitive pairs (sorted by
// magnitude), AB = A - B, same = (A == B).
struct PairInfo {
  int bfA, bfB, prim0, nprim;
  double AB[3];
  int same, pad;
};

struct PairSet {
  const double* prim64;
  const float* prim32;
  const PairInfo* info;
  const float* primdf;
  int npairs;      // shell pairs (records of info)
  int nprimpairs;  // primitive-pair records
};

#define HF_NPAIRCLASS 15  // (la, lb), la >= lb, l <= 4

// One molecule of a launch: density and J/K outputs (device, nbf x nbf
// row-major), its own pair data and ket lists (ket_off[Y] = start of pair
// class Y in ketlist), and whether it takes part (inactive molecules'
// work items are skipped).  Unrestricted (two-spin) builds set Dj (the
// density J is built from, D^a + D^b; null = D), D2 and K2 (the second
// spin's density and exchange): one integral evaluation then feeds J[Dj],
// K[D] and K2[D2].
struct MolJK {
  const double* D;
  double* J;
  double* K;
  int nbf;
  int active;
  PairSet ps;
  const int* ketlist;
  int ket_off[HF_NPAIRCLASS];
  const double* Dj;
  const double* D2;
  double* K2;
};

struct KernelCommon {
  const double* boys64;
  const float* boys32;
  int boys_fp32;  // evaluate F_m in FP32 for reduced-precision quartets
  const float* boysdf;
  int boys_df;    // reduced-precision quartets take F_m from the df64 evaluation (df64 tier)
  int det;        // J/K outputs are fixed-point integer accumulators (deterministic order)
  int* status;    // bounds-checked builds: first failed check (code, then the index), else unused
  const double* rys;  // Rys roots and weights table (rys.cuh layout)
};

// Bounds-checked build (-DHF_BOUNDS_CHECK, small cases in place of a memory
// checker): the J/K kernels test every work-item, pair, primitive-record,
// Boys-row and matrix index before use; a failure stores its check code and
// the offending index in kc.status (first failure wins) and skips the
// access.  The host reads the status after each J/K build.  Without the
// macro the checks compile to nothing.
#ifdef HF_BOUNDS_CHECK
#define HF_BCHECK(kc, ok, code, idx)                                   \
  ((ok) ? true                                                          \
        : (atomicCAS((kc).status, 0, (code)) == 0 ? (void)atomicExch((kc).status + 1, (int)(idx)) : (void)0, false))
#else
#define HF_BCHECK(kc, ok, code, idx) true
#endif
#define HF_BC_ITEM 1   // work-item entry or ket position
#define HF_BC_PAIR 2   // shell-pair id
#define HF_BC_PRIM 3   // primitive-pair record
#define HF_BC_MAT 4    // D/J/K element
#define HF_BC_BOYS 5   // Boys table row

// Work list of one (class, precision) launch.  Entry e pairs bra pair
// bra[e] with the kets ket[kbeg[e] .. kend[e]) of the ket class list
// (significant-primitive-count buckets, Schwarz-descending inside each).
struct JKWork {
  const int* bra;   // [nbra] bra pair ids
  const int* ket;   // ket list of the ket class (single-molecule launches)
  const int* kbeg;  // [nbra] first ket index of each entry
  const int* kend;  // [nbra] one past the last ket index
  const int* ioff;  // [nbra+1] first work item of each entry (32 kets per item, times nsplit)
  const int* mol;   // [nbra] molecule of each entry (multi-molecule launches), else null
  const int* nsplit;  // [nbra] parts each item of the entry is split into along its primitive
                      // loop (bra primitive pairs, or primitive quartets for warp-cooperative
                      // classes); null = 1.  Item t of entry e is ket block (t - ioff[e]) / nsplit[e],
                      // part (t - ioff[e]) % nsplit[e].
  int nbra;
  int nitems;
  int* counter;     // work-item counter, zero before the launch
  int chunk;        // kets per work item (32, or 1 for warp-cooperative classes)
  int nchunk;       // Rys lists: each item's nsplit parts are nchunk output chunks times
                    // ranges of primitive quartets (part = range * nchunk + chunk); 0 otherwise
};

// pair class of (la, lb), la >= lb: ss 0, ps 1, pp 2, ds 3, dp 4, dd 5, fs 6, ... gg 14
__host__ __device__ inline int pair_class(int la, int lb) { return la * (la + 1) / 2 + lb; }
// inverse of pair_class: (la, lb) of pair class X
__host__ __device__ inline void pair_ls(int X, int* la, int* lb) {
  int l = 0;
  while ((l + 1) * (l + 2) / 2 <= X) ++l;
  *la = l;
  *lb = X - l * (l + 1) / 2;
}
__host__ __device__ inline int class_index(int la, int lb, int lc, int ld) {
  const int x = pair_class(la, lb), y = pair_class(lc, ld);
  return x * (x + 1) / 2 + y;
}

// Class launch: grid blocks of `threads` threads (128 = four warps, or 32 =
// one warp per block when a class has few work items) on a stream.
typedef void (*jk_launch_fn)(const JKWork&, const PairSet&, const KernelCommon&, const MolJK&, const MolJK*, int grid,
                             int threads, cudaStream_t);
typedef void (*store_launch_fn)(const JKWork&, const PairSet&, const KernelCommon&, double*, int, int, cudaStream_t);
typedef void (*schwarz_launch_fn)(const int*, int, const PairSet&, const KernelCommon&, double*, cudaStream_t);
typedef int (*occ_fn)();
// Nuclear-gradient launch of one class: the class's Rys work list, the
// density D (nbf x nbf), the atom of every basis function, and the
// gradient accumulator (natom x 3).
typedef void (*grad_launch_fn)(const JKWork&, const PairSet&, const KernelCommon&, const double* D,
                               const int* bf_atom, int nbf, double* grad, int grid, cudaStream_t);

struct EriClassOps {
  jk_launch_fn jk64;
  jk_launch_fn jk32;
  jk_launch_fn jkdf;  // df64 variant
  jk_launch_fn jkrys; // Rys-quadrature route (HF_JK_RYS; the only route of the f/g classes)
  store_launch_fn store;
  schwarz_launch_fn schwarz;
  occ_fn occ64;
  occ_fn occ32;
  occ_fn occdf;
  occ_fn occrys;
  grad_launch_fn grad;  // derivative ERIs contracted for the RHF gradient (Rys route, every class)
  int chunk;      // kets per work item: 32 (warp of quartets) or 1 (warp-cooperative class)
  int rys_nchunks;  // output chunks per quartet of the Rys kernel (every class)
  int rys_native;   // the class has an f or g shell: only the Rys kernel serves it
  int vrr_flops;  // per primitive quartet, as generated
  int hrr_flops;  // per contracted quartet
  const char* name;
};

#ifndef HF_NCLASS
#define HF_NCLASS 120
#endif

// Filled by the per-class translation units.
void hf_register_classes_sp(EriClassOps* table);
void hf_register_classes_d1(EriClassOps* table);
void hf_register_classes_d2(EriClassOps* table);
void hf_register_classes_d3(EriClassOps* table);
void hf_register_classes_d4(EriClassOps* table);
void hf_register_classes_d5(EriClassOps* table);
void hf_register_classes_d6(EriClassOps* table);
// Rys route: every class's jkrys, and all kernels of the f/g classes
void hf_register_classes_rys(EriClassOps* table);
// (rys_thread.cu) thread-per-quartet launchers of the small f/g classes,
// null for the others
void hf_rys_thread_classes(jk_launch_fn* jk, occ_fn* occ);
