/*
 * hf.h -- C ABI of libhf: closed-shell Hartree-Fock two-electron hot path
 * (electron repulsion integrals over contracted Cartesian Gaussians and
 * their contraction into the Coulomb and exchange matrices) on one GPU.
 *
 * Paper: P. Souvatzis, "Uquantchem: a versatile and easy to use quantum
 * chemistry computational software" (arXiv:1303.4916).
 *   Eq. 1      contracted Cartesian Gaussian basis functions
 *   Eqs. 2-4   one-electron matrices S, T, V
 *   Eq. 5      two-electron integrals (ij|kl)
 *   J/K eq.    J_ij = sum_kl (ij|kl) P_kl,  K_il = sum_jk (ij|kl) P_jk
 *              (Sec. "Technical details", the part of HF the paper's MPI
 *              build parallelises)
 *   DIIS       Pulay extrapolation (Sec. "Technical details")
 *
 * Conventions for every entry point:
 *   - Return value: HF_OK (0) on success, a negative HF_ERR_* code on
 *     failure, HF_PENDING (1) only from hf_serve_poll.  hf_strerror()
 *     names a code; hf_last_error() gives the message of the most recent
 *     failure on the calling thread (CUDA error text included).
 *   - Matrices are row-major, double precision, nbf x nbf, where nbf is the
 *     number of Cartesian basis functions ((l+1)(l+2)/2 per shell, shells
 *     in the order given).  Components within a shell: x power from l down
 *     to 0, then y power from l-x down to 0 (p: x,y,z; d: xx,xy,xz,yy,yz,zz).
 *     Every Cartesian component is normalised to unit self-overlap.
 *   - Matrix arguments are DEVICE pointers (e.g. torch CUDA tensors) on the
 *     context's stream unless a flag says HOST.  The caller owns every
 *     buffer it passes; the library owns every handle until its destroy.
 *     Calls are stream-ordered on the context stream and return after the
 *     work is complete unless stated otherwise.
 *   - Coordinates are in bohr, energies in hartree.
 *   - A handle is used by one host thread at a time (the serving loop has
 *     its own worker thread and its own locking).
 */
#ifndef HF_H_
#define HF_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */

#define HF_OK 0
#define HF_PENDING 1
#define HF_ERR_INVALID (-1)        /* bad argument, size or index */
#define HF_ERR_UNSUPPORTED_L (-2)  /* shell angular momentum above HF_LMAX */
#define HF_ERR_OOM (-3)            /* device or host allocation failed */
#define HF_ERR_LINDEP (-4)         /* lambda_min(S) below 1e-10: basis linearly dependent */
#define HF_ERR_NOT_CONVERGED (-5)  /* SCF hit max_iter; the result is still filled */
#define HF_ERR_TIMEOUT (-6)        /* a bounded wait ran out */
#define HF_ERR_CUDA (-7)           /* CUDA / cuBLAS / cuSOLVER call failed */
#define HF_ERR_ODD_ELECTRONS (-8)  /* closed-shell RHF needs an even electron count */
#define HF_ERR_NOT_FOUND (-9)      /* unknown serving ticket */
#define HF_ERR_QUEUE_FULL (-10)    /* serving queue at capacity */
#define HF_ERR_CANCELLED (-11)     /* request cancelled / server shut down */
#define HF_ERR_TOO_LARGE (-12)     /* request footprint exceeds the HBM budget, or a
                                      class's work list exceeds 2^30 items */

#define HF_LMAX 4                  /* highest shell angular momentum (g); quartets with an f or
                                      g shell take the Rys-quadrature route (Eq. 5 by Rys
                                      quadrature, as the paper evaluates it) */
#define HF_MAX_NPRIM 16            /* most primitives in one contracted shell */
#define HF_STORED_NBF_MAX 400      /* largest nbf of the stored-tensor calls (nbf^4 doubles:
                                      205 GB at 400, held in HBM) */

/* ---------------------------------------------------------------- types */

typedef struct hf_ctx hf_ctx;
typedef struct hf_basis hf_basis;
typedef struct hf_server hf_server;

/* One nucleus: charge Z and position (bohr). */
typedef struct {
    int Z;
    double xyz[3];
} hf_atom;

/* One contracted shell (Eq. 1): centre atom, angular momentum l (0..4),
 * nprim primitives starting at exps[prim_off], coefs[prim_off].  The
 * coefficients d_n multiply normalised primitives; the library rescales
 * the contraction to unit norm. */
typedef struct {
    int atom;
    int l;
    int nprim;
    int prim_off;
} hf_shell;

/* J/K build options.  hf_jk_opts_default() fills the defaults shown. */
#define HF_JK_HOST 1u              /* D, J, K are host pointers: copies are done inside the call */
#define HF_JK_DETERMINISTIC 2u     /* bitwise reproducible J, K: contributions accumulate as
                                      fixed-point integers (units 2^-20 and 2^-56 per
                                      element, order-independent) instead of FP64 atomics;
                                      hf_fock_jk, hf_fock_jk_profiled and hf_fock_jk_uhf
                                      only (the basis keeps 32 bytes of device scratch per
                                      matrix element, 48 for hf_fock_jk_uhf); the SCF,
                                      batch, serving and no-alloc calls reject it */
#define HF_JK_FP32_BOYS 4u         /* reduced-precision quartets also evaluate F_m(T) in FP32 */
#define HF_JK_DF64 8u              /* quartets above fp32_bound run in double-float (FP32-pair)
                                      arithmetic, ~1e-14 relative, in every class (J/K
                                      digestion and accumulation stay FP64) */
#define HF_JK_RYS 16u              /* every class by Rys quadrature (Eq. 5, the paper's route) in
                                      FP64, in place of the Obara-Saika / Head-Gordon-Pople
                                      kernels of the s/p/d classes; classes with an f or g shell
                                      always take it (in FP64 also under HF_JK_DF64 and for
                                      quartets below fp32_bound) */
typedef struct {
    double schwarz_tau;  /* drop shell quartet iff Q_ab*Q_cd < tau (default 1e-12; 0 keeps all) */
    double fp32_bound;   /* quartets with Q_ab*Q_cd < fp32_bound run in FP32 (default 0 = none) */
    unsigned flags;      /* HF_JK_* */
} hf_jk_opts;

/* SCF options.  hf_scf_opts_default() fills the defaults shown. */
#define HF_SCF_STORED_ERI 1u       /* build the N^4 ERI tensor once and contract it
                                      (nbf <= HF_STORED_NBF_MAX, device memory permitting) */
typedef struct {
    int max_iter;        /* default 128 */
    double e_tol;        /* stop when |E_k - E_{k-1}| <= e_tol (default 1e-8) */
    int diis_size;       /* Pulay DIIS subspace, 0 = off (default 8, at most 16) */
    const double* D0;    /* optional initial density (device, nbf x nbf); NULL = core guess */
    hf_jk_opts jk;
    unsigned flags;      /* HF_SCF_* */
} hf_scf_opts;

/* SCF result.  The caller may point D, C, eps, F, F1 at DEVICE buffers
 * (nbf x nbf, or nbf for eps) to receive them; NULL skips an output. */
typedef struct {
    double energy;       /* total energy E = Tr[D(H+F)] + E_nuc */
    double e_elec;
    double e_nuc;
    double delta_e;      /* |E_k - E_{k-1}| at the last iteration */
    double diis_error;   /* max |F D S - S D F| at the last iteration */
    double homo_lumo_gap;
    int iterations;
    int converged;
    long long fock_builds;
    long long quartets;  /* shell quartets evaluated over all builds */
    double seconds;      /* wall time of the solve */
    double* D;
    double* C;
    double* eps;
    double* F;           /* last Fock matrix before DIIS extrapolation */
    double* F1;          /* Fock matrix of iteration 1, F(D_1) */
} hf_scf_result;

void hf_jk_opts_default(hf_jk_opts* o);
void hf_scf_opts_default(hf_scf_opts* o);
const char* hf_strerror(int code);
const char* hf_last_error(void);

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device`.  hbm_budget (bytes) caps the
 * device memory the serving loop admits work into (0 = 80% of free
 * memory).  cuda_stream is a cudaStream_t to use (NULL = the library
 * creates its own stream, ordered after the legacy default stream).  Errors: HF_ERR_INVALID,
 * HF_ERR_CUDA (no device), HF_ERR_OOM. */
int hf_ctx_create(hf_ctx** out, int device, size_t hbm_budget, void* cuda_stream);
/* Destroy a context.  Bases and servers created on it and not yet
 * destroyed keep it alive: the last hf_basis_destroy or hf_serve_destroy
 * completes the teardown (no new basis may be created on it meanwhile:
 * HF_ERR_INVALID). */
void hf_ctx_destroy(hf_ctx* ctx);
/* The stream all work of this context is ordered on (a cudaStream_t). */
void* hf_ctx_stream(hf_ctx* ctx);
/* Number of SMs of the context's device. */
int hf_ctx_num_sms(hf_ctx* ctx);

/* Log every SCF iteration of this context (hf_scf_solve, hf_uhf_solve,
 * hf_scf_solve_batch, serving) as one JSON line appended to the file
 * `path` ("-" = stderr, NULL = logging off, the default):
 *   {"event": "scf_iter", "solver": "rhf"|"uhf"|"batch"|"serve", "mol": tag,
 *    "nbf": n, "iter": k, "energy": E_k, "delta_e": |E_k - E_{k-1}| or null,
 *    "diis_error": max |F D S - S D F|, "t": seconds since the solve began,
 *    "converged": 0|1}
 * Errors: HF_ERR_INVALID (null context, file cannot be opened). */
int hf_ctx_set_log(hf_ctx* ctx, const char* path);

/* 1 when the library was built with -DHF_BOUNDS_CHECK (every index of the
 * J/K kernels checked before use, a failure returned as HF_ERR_INVALID
 * naming the index; for small test cases), else 0. */
int hf_bounds_checked(void);

/* Fault-injection hook for tests: make the n-th device allocation from now
 * on fail with HF_ERR_OOM (n >= 1); n = 0 disables.  Host-side only. */
void hf_ctx_inject_alloc_failure(hf_ctx* ctx, int n);

/* ---------------------------------------------------------------- basis */

/* Build the device-resident basis of one molecule: normalised contraction
 * coefficients (Eq. 1), shell-pair data (Gaussian product centres and
 * prefactors per primitive pair), Schwarz factors Q_ab and the
 * class-bucketed quartet work lists.  All input arrays are host memory and
 * are copied.  n_electrons >= 0 is the count the closed-shell calls use
 * (hf_scf_solve and hf_scf_solve_batch return HF_ERR_ODD_ELECTRONS for an
 * odd one; hf_uhf_solve takes its own spin counts).
 * Errors: HF_ERR_INVALID (also a shell with more than HF_MAX_NPRIM
 * primitives, a contraction of zero norm, two charged atoms at one point),
 * HF_ERR_UNSUPPORTED_L (l > HF_LMAX), HF_ERR_OOM, HF_ERR_CUDA. */
int hf_basis_create(hf_ctx* ctx, const hf_atom* atoms, int natom, const hf_shell* shells,
                    int nshell, const double* exps, const double* coefs, int n_electrons,
                    hf_basis** out);
void hf_basis_destroy(hf_basis* b);
int hf_basis_nbf(const hf_basis* b);
int hf_basis_nshell(const hf_basis* b);
/* Device bytes held by the basis handle. */
size_t hf_basis_device_bytes(const hf_basis* b);

/* Schwarz factors Q_ab = sqrt(max_{a in A, b in B} |(ab|ab)|) for all shell
 * pairs, nshell x nshell row-major, written to HOST memory Q.  The
 * screening rule itself is not in the paper; it is the standard bound
 * |(ab|cd)| <= Q_ab Q_cd on Eq. 5. */
int hf_schwarz(hf_basis* b, double* Q_host);

/* Shell quartets the J/K build evaluates for the given options: unique
 * under the 8-fold symmetry of Eq. 5 and surviving Schwarz screening.
 * n_fp32 (may be NULL) receives how many of them run in FP32. */
int hf_count_quartets(hf_basis* b, const hf_jk_opts* opts, long long* n_total, long long* n_fp32);

/* The J/K contraction (Sec. "Technical details", J/K equation) for a
 * symmetric density P = D:  J_ij = sum_kl (ij|kl) D_kl,
 * K_il = sum_jk (ij|kl) D_jk.  D, J, K are nbf x nbf, device pointers
 * (host pointers with HF_JK_HOST).  J and K are overwritten.  opts may be
 * NULL (defaults).  Errors: HF_ERR_INVALID, HF_ERR_CUDA, HF_ERR_OOM,
 * HF_ERR_TOO_LARGE (an angular class with more than 2^30 work items). */
int hf_fock_jk(hf_basis* b, const double* D, double* J, double* K, const hf_jk_opts* opts);

/* Work statistics of one canonical class (la lb | lc ld), for roofline
 * accounting: unique surviving shell quartets and primitive quartets
 * (after primitive-pair screening) in each precision, and the generated
 * operation counts of the class's recurrences. */
#define HF_NCLASS 120             /* (la lb | lc ld) with l <= 4, pair classes ordered */
typedef struct {
    int la, lb, lc, ld;
    int vrr_flops;           /* VRR operations per primitive quartet */
    int hrr_flops;           /* HRR operations per contracted quartet */
    int prim_flops;          /* total operations per primitive quartet (setup + Boys + VRR) */
    int digest_flops;        /* J/K digestion operations per contracted quartet */
    long long quartets_fp64, prim_quartets_fp64;
    long long quartets_fp32, prim_quartets_fp32;
} hf_class_stats;
int hf_class_stats_get(hf_basis* b, const hf_jk_opts* opts, hf_class_stats* out /* HF_NCLASS entries */);

/* hf_fock_jk with a CUDA-event timing of every class kernel on the
 * context stream: class_ms[2*c] (FP64) and class_ms[2*c+1] (FP32) receive
 * the duration of class c's launch in milliseconds (0 when not launched).
 * Device pointers only. */
int hf_fock_jk_profiled(hf_basis* b, const double* D, double* J, double* K, const hf_jk_opts* opts,
                        double* class_ms);

/* hf_fock_jk for callers that cannot allocate device memory.  The paper
 * has no counterpart: it is a deployment form of the J/K build above for
 * code where cudaMalloc is off limits when the Fock build runs (a frozen
 * allocator, a host framework that owns all device memory, a real-time
 * loop).  Same inputs, outputs, precision tiers (HF_JK_DF64,
 * HF_JK_FP32_BOYS, fp32_bound) and results as hf_fock_jk, device pointers
 * only; the J'/K' accumulators and work-item counters live in one static
 * device array of the library, so the call allocates nothing.
 * Limits: nbf <= 512 (HF_ERR_TOO_LARGE above); about 4 MiB of static device
 * memory is held on every GPU that loads the library until exit.
 * The first call on a device looks up the array's address (once per
 * device): make it before any stream capture, and do not use the entry
 * point on a device after cudaDeviceReset.  All calls share the array, so
 * calls that overlap on the GPU race.  The quartet work lists for the
 * options must already exist on the basis (a prior hf_fock_jk or
 * hf_count_quartets with the same options), else HF_ERR_INVALID; a
 * negative threshold is HF_ERR_INVALID as in hf_fock_jk. */
int hf_fock_jk_noalloc(hf_basis* b, const double* D, double* J, double* K, const hf_jk_opts* opts);

/* One-electron matrices of Eqs. 2-4 (device pointers, any may be NULL)
 * and the nuclear repulsion energy (host, may be NULL). */
int hf_one_electron(hf_basis* b, double* S, double* T, double* V, double* e_nuc);

/* Full ERI tensor G[i][j][k][l] = (ij|kl) of Eq. 5 into a DEVICE buffer of
 * nbf^4 doubles (nbf <= HF_STORED_NBF_MAX; the caller allocates it).
 * Errors: HF_ERR_INVALID. */
int hf_eri_tensor(hf_basis* b, double* G);

/* J and K from a stored ERI tensor G (device, nbf^4): J = G vec(D),
 * K_il = sum_jk G_ijkl D_jk.  Same contract as hf_fock_jk otherwise. */
int hf_jk_stored(hf_basis* b, const double* G, const double* D, double* J, double* K);

/* Closed-shell RHF (Szabo-Ostlund procedure; DIIS of Pulay): Loewdin
 * X = S^{-1/2}, core guess, then per iteration diagonalise X^T F X,
 * D = C_occ C_occ^T, J/K of D, F = H + 2J - K, E = Tr[D(H+F)] + E_nuc,
 * DIIS with error F D S - S D F, until |dE| <= e_tol.  The J/K phase of an
 * iteration is captured once into a CUDA graph and replayed.
 * Returns HF_ERR_NOT_CONVERGED (result filled) after max_iter,
 * HF_ERR_LINDEP if lambda_min(S) < 1e-10, HF_ERR_ODD_ELECTRONS for an odd
 * electron count of the basis. */
int hf_scf_solve(hf_basis* b, const hf_scf_opts* opts, hf_scf_result* res);

/* ---------------------------------------------------------------- unrestricted */

/* Unrestricted (two-spin) J/K, the contraction of the J/K equation
 * (Sec. "Technical details") as the paper's UHF calculations need it:
 * J = J[Da + Db], Ka = K[Da], Kb = K[Db], all three from one evaluation of
 * the integrals of Eq. 5.  Da, Db, J, Ka, Kb are nbf x nbf DEVICE pointers
 * (symmetric densities; the outputs are overwritten).  opts as for
 * hf_fock_jk except HF_JK_HOST (HF_ERR_INVALID).  The basis keeps one
 * nbf x nbf device buffer for Da + Db after the first call.  Errors as
 * hf_fock_jk. */
int hf_fock_jk_uhf(hf_basis* b, const double* Da, const double* Db, double* J, double* Ka, double* Kb,
                   const hf_jk_opts* opts);

/* UHF result.  Da, Db (nbf x nbf) and eps_a, eps_b (nbf) may point at
 * DEVICE buffers to receive the converged spin densities and orbital
 * energies; NULL skips an output. */
typedef struct {
    double energy;       /* E = (1/2) sum_s Tr[D^s (H + F^s)] + E_nuc */
    double e_elec;
    double e_nuc;
    double delta_e;      /* |E_k - E_{k-1}| at the last iteration */
    double diis_error;   /* max |F^s D^s S - S D^s F^s| over both spins */
    double s2;           /* <S^2> of the determinant */
    int iterations;
    int converged;
    long long fock_builds;
    long long quartets;
    double seconds;
    double* Da;
    double* Db;
    double* eps_a;
    double* eps_b;
} hf_uhf_result;

/* Unrestricted HF, the form of the paper's test calculations (Sec. "Tests",
 * runs RUN1 and RUN7), by the Pople-Nesbet equations as Szabo-Ostlund state
 * them: per spin s with n_s electrons D^s = C^s_occ C^s_occ^T and
 * F^s = H + J[D^a + D^b] - K[D^s]; Loewdin X, core guess F^a = F^b = H;
 * DIIS (Pulay) on the stacked errors F^s D^s S - S D^s F^s with one set of
 * coefficients for both spins; stop at |E_k - E_{k-1}| <= e_tol.  J, K^a,
 * K^b of an iteration come from one integral evaluation (hf_fock_jk_uhf),
 * replayed from a CUDA graph.  nbf >= n_alpha >= n_beta >= 0; the basis's
 * n_electrons is not used.  opts: as hf_scf_solve without
 * HF_SCF_STORED_ERI and D0 (HF_ERR_INVALID).  Returns HF_ERR_NOT_CONVERGED
 * (result filled) after max_iter, HF_ERR_LINDEP as hf_scf_solve. */
int hf_uhf_solve(hf_basis* b, int n_alpha, int n_beta, const hf_scf_opts* opts, hf_uhf_result* res);

/* ---------------------------------------------------------------- MP2 */

/* Second-order Moller-Plesset correlation energy of a closed-shell RHF
 * solution, the paper's MP2 (Sec. "Capabilities"; its MP2 follows
 * Szabo-Ostlund):
 *   E(2) = sum_{i,j occ} sum_{a,b virt} (ia|jb) [2 (ia|jb) - (ib|ja)]
 *                                        / (e_i + e_j - e_a - e_b)
 * over the canonical orbitals, (ia|jb) from the stored AO tensor of Eq. 5
 * by four one-index transformations (nbf <= HF_STORED_NBF_MAX; the call
 * allocates nbf^4 + nbf^3 n_occ + nbf^2 n_occ n_virt doubles of device memory
 * while it runs, 30 GB at nbf 220, and returns HF_ERR_OOM when they do not
 * fit).
 * C: nbf x nbf DEVICE, row-major, C[mu][p] = coefficient of AO mu in MO p
 * (as hf_scf_result.C); eps: nbf orbital energies, ascending, DEVICE;
 * n_occ in [1, nbf).  *e2 (host) receives E(2).  Errors: HF_ERR_INVALID,
 * HF_ERR_OOM, HF_ERR_CUDA. */
int hf_mp2_energy(hf_basis* b, const double* C, const double* eps, int n_occ, double* e2);

/* ---------------------------------------------------------------- forces */

/* Analytic nuclear gradient dE/dR (natom x 3, Eh/bohr) of the converged
 * closed-shell RHF energy; the paper's Hartree-Fock interatomic forces are
 * its negative.  With D = C_occ C_occ^T and W = C_occ diag(eps_occ)
 * C_occ^T:
 *   dE/dR = 2 sum D dH/dR - 2 sum W dS/dR
 *         + sum_(ijkl) (2 D_ij D_kl - D_ik D_jl) d(ij|kl)/dR + dE_nuc/dR,
 * the derivative integrals of Eq. 5 by Rys quadrature (every class), those
 * of Eqs. 2-4 by Obara-Saika (overlap, kinetic) and Rys quadrature
 * (nuclear attraction, including the derivative of the operator's centre).
 * C: nbf x nbf DEVICE, row-major, C[mu][p] (as hf_scf_result.C); eps: nbf
 * orbital energies, ascending, DEVICE; n_occ occupied orbitals (nelec / 2);
 * opts: Schwarz tau of the derivative quartets (NULL = defaults;
 * HF_JK_HOST and HF_JK_DETERMINISTIC are rejected).  grad: natom x 3 HOST
 * doubles, overwritten.  The call allocates O(nbf^2) device scratch and
 * leaves the basis's work lists in their Rys shape.  Errors:
 * HF_ERR_INVALID, HF_ERR_OOM, HF_ERR_CUDA. */
int hf_rhf_gradient(hf_basis* b, const double* C, const double* eps, int n_occ, const hf_jk_opts* opts,
                    double* grad);

/* ---------------------------------------------------------------- Rys rule */

/* The n-point Rys quadrature rule at T (Eq. 5 evaluated by Rys quadrature):
 * roots u_i = t_i^2 (ascending) and weights w_i with
 *   int_0^1 f(t^2) exp(-T t^2) dt = sum_i w_i f(u_i)
 * exact for polynomials f of degree <= 2n - 1 (so sum_i w_i u_i^k = F_k(T),
 * the Boys function, for k < 2n), from the same table the ERI kernels use
 * (piecewise Chebyshev series for T < 60, the Gauss-Hermite limit above;
 * about 1e-15 relative).  Host only, no device needed.  n in [1, 9];
 * T finite and >= 0; u, w host arrays of n doubles.  Errors:
 * HF_ERR_INVALID. */
int hf_rys_rule(int n, double T, double* u, double* w);

/* ---------------------------------------------------------------- batch */

/* Solve many independent molecules together: each SCF iteration runs one
 * launch per angular class over the quartets of every still-active
 * molecule.  bases[i] must share one context.  opts applies to all;
 * results[i] receives molecule i (its output pointers as in
 * hf_scf_result).  status[i] gets the per-molecule code. */
int hf_scf_solve_batch(hf_basis* const* bases, int count, const hf_scf_opts* opts,
                       hf_scf_result* results, int* status);

/* ---------------------------------------------------------------- serving */

typedef struct {
    int max_active;          /* molecules iterated together (default 64) */
    int queue_capacity;      /* pending requests accepted (default 100000) */
    size_t hbm_budget;       /* bytes of device memory for admitted work (0 = context budget) */
    hf_scf_opts scf;         /* per-request SCF options */
} hf_serve_opts;

typedef struct {
    const hf_atom* atoms;
    int natom;
    const hf_shell* shells;
    int nshell;
    const double* exps;
    const double* coefs;
    int nprim;               /* total primitives (length of exps / coefs) */
    int n_electrons;
} hf_request;

typedef struct {
    int status;              /* HF_OK, HF_ERR_NOT_CONVERGED, ... */
    double energy;
    int iterations;
    int converged;
    int nbf;
    double t_submit;         /* seconds on the server clock */
    double t_admit;
    double t_done;
    long long fock_builds;
    long long quartets;
} hf_serve_result;

void hf_serve_opts_default(hf_serve_opts* o);
/* Start a serving loop on ctx (a worker thread that owns the GPU work).
 * Requests are admitted while their device footprint (pair data, density,
 * Fock, J, K, DIIS history) fits the budget and fewer than max_active are
 * in flight; active molecules advance one SCF iteration per round, newly
 * admitted ones join at the next round, converged ones retire. */
int hf_serve_create(hf_ctx* ctx, const hf_serve_opts* opts, hf_server** out);
/* Copy a request into the queue; *ticket identifies it.  Errors:
 * HF_ERR_INVALID, HF_ERR_QUEUE_FULL, HF_ERR_TOO_LARGE, HF_ERR_CANCELLED. */
int hf_serve_submit(hf_server* s, const hf_request* req, uint64_t* ticket);
/* HF_PENDING while queued or running; HF_OK (result filled, ticket
 * released) when done, including a failed solve whose code is in
 * result->status; HF_ERR_NOT_FOUND for an unknown or released ticket. */
int hf_serve_poll(hf_server* s, uint64_t ticket, hf_serve_result* result);
/* Cancel a queued (not yet admitted) request: HF_OK, or HF_ERR_NOT_FOUND. */
int hf_serve_cancel(hf_server* s, uint64_t ticket);
/* Server clock (seconds since hf_serve_create). */
double hf_serve_now(hf_server* s);
/* Block until every submitted request is done (or timeout_s passes:
 * HF_ERR_TIMEOUT). */
int hf_serve_drain(hf_server* s, double timeout_s);
void hf_serve_destroy(hf_server* s);

#ifdef __cplusplus
}
#endif

#endif /* HF_H_ */
