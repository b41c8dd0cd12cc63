/*
 * hf_oracle.c -- plain, slow CPU oracle for closed-shell Hartree-Fock
 * integrals and the Coulomb / exchange contraction.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library path may link, load or
 * call this file; only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark do.  It shares no code, header, table or constant with
 * the CUDA library.
 *
 * What it computes (all in double precision, long double where noted):
 *   - contracted Cartesian Gaussian basis functions, Eq. 1, each Cartesian
 *     component normalised to unit self-overlap;
 *   - S, T (Eqs. 2-3) by the binomial-expansion (Taylor / Cook) formulas;
 *   - V (Eq. 4) by the McMurchie-Davidson Hermite expansion;
 *   - electron repulsion integrals (ij|kl), Eq. 5, by McMurchie-Davidson
 *     (deliberately neither the paper's Rys route nor the GPU's
 *     Obara-Saika / Head-Gordon-Pople route: all three are exact for the
 *     same quantity);
 *   - J_ij = sum_kl (ij|kl) P_kl and K_il = sum_jk (ij|kl) P_jk, the
 *     contraction of Sec. "Technical details" (J/K equation), with P the
 *     density passed in, no factors applied;
 *   - the Boys function F_m(T) = int_0^1 t^{2m} exp(-T t^2) dt by its power
 *     series in long double (T < 30) or erf plus upward recursion (T >= 30).
 *
 * Cartesian component order within a shell of angular momentum l: x power
 * from l down to 0, then y power from l-x down to 0 (p: x,y,z;
 * d: xx,xy,xz,yy,yz,zz).  Basis functions are numbered shell by shell.
 *
 * Optional Schwarz screening (tau > 0): a shell quartet (AB|CD) is dropped
 * iff Q_AB * Q_CD < tau with Q_AB = sqrt(max over components |(ab|ab)|),
 * computed here from the oracle's own integrals.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_LMAX 4                    /* highest shell l the oracle accepts */
#define OR_LTOT (4 * OR_LMAX)        /* highest total l of a quartet */
#define OR_NCART(l) (((l) + 1) * ((l) + 2) / 2)
#define OR_MAXCART OR_NCART(OR_LMAX)

static const double OR_PI = 3.14159265358979323846264338327950288;

/* ------------------------------------------------------------------ */
/* Boys function                                                        */
/* ------------------------------------------------------------------ */

/* F_m(T) for one m: the Boys function through which the Gaussian integrals
 * of Eqs. 4-5 are expressed.  T < 30: e^{-T} sum_i (2T)^i / prod_{k=0..i} (2m+2k+1),
 * summed in long double until the term is below 1e-22 of the sum.
 * T >= 30: F_0 = (1/2) sqrt(pi/T) erf(sqrt T), then upward recursion
 * F_{k+1} = ((2k+1) F_k - e^{-T}) / (2T). */
double or_boys(int m, double T)
{
    if (T < 30.0) {
        long double t = (long double)T;
        long double term = 1.0L / (long double)(2 * m + 1);
        long double sum = term;
        for (int i = 1; i < 2000; ++i) {
            term *= 2.0L * t / (long double)(2 * m + 2 * i + 1);
            sum += term;
            if (term < 1e-22L * sum) break;
        }
        return (double)(expl(-t) * sum);
    }
    long double t = (long double)T;
    long double f = 0.5L * sqrtl((long double)OR_PI / t) * erfl(sqrtl(t));
    long double et = expl(-t);
    for (int k = 0; k < m; ++k) f = ((2 * k + 1) * f - et) / (2.0L * t);
    return (double)f;
}

/* ------------------------------------------------------------------ */
/* Basis                                                                */
/* ------------------------------------------------------------------ */

typedef struct {
    int natom;
    int *Z;
    double *xyz;            /* natom x 3 */
    int nshell;
    int *sh_atom, *sh_l, *sh_nprim, *sh_prim, *sh_bf;
    double *exps;           /* primitive exponents */
    int nbf;
    int *bf_shell;          /* shell of each basis function */
    int *bf_lmn;            /* nbf x 3 Cartesian powers */
    double *bf_coef;        /* per bf, per primitive of its shell: d_k N_k c */
    int *bf_coef_off;       /* offset of each bf's coefficients */
} or_basis;

static double dfact(int n) /* (n)!! with (-1)!! = 1 */
{
    double r = 1.0;
    for (int k = n; k > 1; k -= 2) r *= k;
    return r;
}

static void cart_powers(int l, int idx, int *lx, int *ly, int *lz)
{
    int c = 0;
    for (int x = l; x >= 0; --x)
        for (int y = l - x; y >= 0; --y) {
            if (c == idx) { *lx = x; *ly = y; *lz = l - x - y; return; }
            ++c;
        }
}

/* Primitive normalisation of x^a y^b z^c exp(-alpha r^2) (the Gaussians of Eq. 1). */
static double prim_norm(double alpha, int a, int b, int c)
{
    int L = a + b + c;
    double n2 = pow(2.0 * alpha / OR_PI, 1.5) * pow(4.0 * alpha, L) /
                (dfact(2 * a - 1) * dfact(2 * b - 1) * dfact(2 * c - 1));
    return sqrt(n2);
}

/* Overlap of two unnormalised primitives x^a.. on the SAME centre. */
static double same_centre_overlap(double p, int a, int b, int c)
{
    return pow(OR_PI / p, 1.5) * dfact(2 * a - 1) * dfact(2 * b - 1) * dfact(2 * c - 1) /
           pow(2.0 * p, a + b + c);
}

void or_basis_free(or_basis *B)
{
    if (!B) return;
    free(B->Z); free(B->xyz); free(B->sh_atom); free(B->sh_l); free(B->sh_nprim);
    free(B->sh_prim); free(B->sh_bf); free(B->exps); free(B->bf_shell); free(B->bf_lmn);
    free(B->bf_coef); free(B->bf_coef_off); free(B);
}

/* Contracted basis of Eq. 1: each Cartesian component sum_k d_k N_k g_k,
 * rescaled to unit self-overlap.  Returns NULL on invalid input (l > OR_LMAX,
 * nprim < 1, bad index). */
or_basis *or_basis_new(int natom, const int *Z, const double *xyz, int nshell,
                       const int *sh_atom, const int *sh_l, const int *sh_nprim,
                       const int *sh_prim, int nprim_total, const double *exps,
                       const double *coefs)
{
    or_basis *B = (or_basis *)calloc(1, sizeof(or_basis));
    B->natom = natom;
    B->Z = (int *)malloc(sizeof(int) * (natom > 0 ? natom : 1));
    B->xyz = (double *)malloc(sizeof(double) * 3 * (natom > 0 ? natom : 1));
    memcpy(B->Z, Z, sizeof(int) * natom);
    memcpy(B->xyz, xyz, sizeof(double) * 3 * natom);
    B->nshell = nshell;
    B->sh_atom = (int *)malloc(sizeof(int) * nshell);
    B->sh_l = (int *)malloc(sizeof(int) * nshell);
    B->sh_nprim = (int *)malloc(sizeof(int) * nshell);
    B->sh_prim = (int *)malloc(sizeof(int) * nshell);
    B->sh_bf = (int *)malloc(sizeof(int) * (nshell + 1));
    B->exps = (double *)malloc(sizeof(double) * nprim_total);
    memcpy(B->sh_atom, sh_atom, sizeof(int) * nshell);
    memcpy(B->sh_l, sh_l, sizeof(int) * nshell);
    memcpy(B->sh_nprim, sh_nprim, sizeof(int) * nshell);
    memcpy(B->sh_prim, sh_prim, sizeof(int) * nshell);
    memcpy(B->exps, exps, sizeof(double) * nprim_total);
    int nbf = 0, ncoef = 0;
    for (int s = 0; s < nshell; ++s) {
        if (sh_l[s] < 0 || sh_l[s] > OR_LMAX || sh_nprim[s] < 1 || sh_atom[s] < 0 ||
            sh_atom[s] >= natom || sh_prim[s] < 0 || sh_prim[s] + sh_nprim[s] > nprim_total) {
            or_basis_free(B);
            return NULL;
        }
        B->sh_bf[s] = nbf;
        nbf += OR_NCART(sh_l[s]);
        ncoef += OR_NCART(sh_l[s]) * sh_nprim[s];
    }
    B->sh_bf[nshell] = nbf;
    B->nbf = nbf;
    B->bf_shell = (int *)malloc(sizeof(int) * nbf);
    B->bf_lmn = (int *)malloc(sizeof(int) * 3 * nbf);
    B->bf_coef = (double *)malloc(sizeof(double) * ncoef);
    B->bf_coef_off = (int *)malloc(sizeof(int) * nbf);
    int co = 0;
    for (int s = 0; s < nshell; ++s) {
        int l = sh_l[s], K = sh_nprim[s], p0 = sh_prim[s];
        for (int c = 0; c < OR_NCART(l); ++c) {
            int bf = B->sh_bf[s] + c, a = 0, b = 0, cc = 0;
            cart_powers(l, c, &a, &b, &cc);
            B->bf_shell[bf] = s;
            B->bf_lmn[3 * bf] = a; B->bf_lmn[3 * bf + 1] = b; B->bf_lmn[3 * bf + 2] = cc;
            B->bf_coef_off[bf] = co;
            /* d_k N_k for this Cartesian component */
            for (int k = 0; k < K; ++k)
                B->bf_coef[co + k] = coefs[p0 + k] * prim_norm(exps[p0 + k], a, b, cc);
            /* rescale so that <phi|phi> = 1 (Eq. 1 functions, unit norm) */
            double self = 0.0;
            for (int k = 0; k < K; ++k)
                for (int k2 = 0; k2 < K; ++k2)
                    self += B->bf_coef[co + k] * B->bf_coef[co + k2] *
                            same_centre_overlap(exps[p0 + k] + exps[p0 + k2], a, b, cc);
            double f = 1.0 / sqrt(self);
            for (int k = 0; k < K; ++k) B->bf_coef[co + k] *= f;
            co += K;
        }
    }
    return B;
}

int or_basis_nbf(const or_basis *B) { return B->nbf; }

/* first basis function of each shell, nshell+1 entries */
void or_basis_shell_bf(const or_basis *B, int *out)
{
    memcpy(out, B->sh_bf, sizeof(int) * (B->nshell + 1));
}

static const double *centre(const or_basis *B, int shell)
{
    return B->xyz + 3 * B->sh_atom[shell];
}

/* ------------------------------------------------------------------ */
/* One-electron integrals                                               */
/* ------------------------------------------------------------------ */

static double binom(int n, int k)
{
    double r = 1.0;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}

/* Overlap integrals, Eq. 2.  1D factor of (x-A)^la (x-B)^lb exp(-p (x-P)^2) by binomial
 * expansion about P: sum_ij C(la,i) C(lb,j) PA^{la-i} PB^{lb-j}
 * int u^{i+j} e^{-p u^2} du. */
static double tho_overlap_1d(int la, int lb, double PA, double PB, double p)
{
    double s = 0.0;
    for (int i = 0; i <= la; ++i)
        for (int j = 0; j <= lb; ++j) {
            int n = i + j;
            if (n % 2) continue;
            double mom = dfact(n - 1) / pow(2.0 * p, n / 2) * sqrt(OR_PI / p);
            s += binom(la, i) * binom(lb, j) * pow(PA, la - i) * pow(PB, lb - j) * mom;
        }
    return s;
}

/* Overlap of two unnormalised Cartesian primitives. */
static double prim_overlap(double a, const double *A, const int *la, double b,
                           const double *B, const int *lb)
{
    double p = a + b, mu = a * b / p, r2 = 0.0, s = 1.0;
    for (int x = 0; x < 3; ++x) {
        double P = (a * A[x] + b * B[x]) / p;
        r2 += (A[x] - B[x]) * (A[x] - B[x]);
        s *= tho_overlap_1d(la[x], lb[x], P - A[x], P - B[x], p);
    }
    return exp(-mu * r2) * s;
}

/* Kinetic energy integrals, Eq. 3, of two primitives: the ket is differentiated,
 * -1/2 <a|nabla^2|b> = b(2(lx+ly+lz)+3) <a|b> - 2 b^2 sum_x <a|b+2_x>
 *                      - 1/2 sum_x lx(lx-1) <a|b-2_x>. */
static double prim_kinetic(double a, const double *A, const int *la, double b,
                           const double *B, const int *lb)
{
    int L = lb[0] + lb[1] + lb[2];
    double t = b * (2 * L + 3) * prim_overlap(a, A, la, b, B, lb);
    for (int x = 0; x < 3; ++x) {
        int up[3] = {lb[0], lb[1], lb[2]};
        up[x] += 2;
        t -= 2.0 * b * b * prim_overlap(a, A, la, b, B, up);
        if (lb[x] >= 2) {
            int dn[3] = {lb[0], lb[1], lb[2]};
            dn[x] -= 2;
            t -= 0.5 * lb[x] * (lb[x] - 1) * prim_overlap(a, A, la, b, B, dn);
        }
    }
    return t;
}

/* McMurchie-Davidson Hermite expansion coefficients for one axis:
 * E[i][j][t], i <= la, j <= lb, t <= i+j, with E^{00}_0 = 1 (the Gaussian
 * product exponential is applied by the caller). */
#define EDIM (OR_LMAX + 3)
static void hermite_E(int la, int lb, double PA, double PB, double oo2p,
                      double E[EDIM][EDIM][2 * EDIM])
{
    memset(E, 0, sizeof(double) * EDIM * EDIM * 2 * EDIM);
    E[0][0][0] = 1.0;
    for (int i = 0; i < la; ++i)
        for (int t = 0; t <= i + 1; ++t) {
            double v = PA * E[i][0][t];
            if (t > 0) v += oo2p * E[i][0][t - 1];
            if (t + 1 <= i) v += (t + 1) * E[i][0][t + 1];
            E[i + 1][0][t] = v;
        }
    for (int i = 0; i <= la; ++i)
        for (int j = 0; j < lb; ++j)
            for (int t = 0; t <= i + j + 1; ++t) {
                double v = PB * E[i][j][t];
                if (t > 0) v += oo2p * E[i][j][t - 1];
                if (t + 1 <= i + j) v += (t + 1) * E[i][j][t + 1];
                E[i][j + 1][t] = v;
            }
}

/* Scratch for one thread: Hermite tables of one primitive quartet. */
#define RD (OR_LTOT + 1)
typedef struct {
    double Rw[RD][RD][RD][RD];          /* R^n_{tuv} for all n */
    double R[RD * RD * RD];             /* R^0_{tuv} */
    double Eab[3][EDIM][EDIM][2 * EDIM];
    double Ecd[3][EDIM][EDIM][2 * EDIM];
} or_ws;

static or_ws *ws_new(void) { return (or_ws *)malloc(sizeof(or_ws)); }

/* Hermite Coulomb integrals R^0_{tuv}(alpha, X, Y, Z) for t+u+v <= L,
 * from R^n_{000} = (-2 alpha)^n F_n(alpha |XYZ|^2) and
 * R^n_{t+1,u,v} = t R^{n+1}_{t-1,u,v} + X R^{n+1}_{t,u,v} (same for u, v).
 * Stored as R[t][u][v] with dimension RD. */
static void hermite_R(or_ws *ws, int L, double alpha, double X, double Y, double Z, double *Rout)
{
    double (*work)[RD][RD][RD] = ws->Rw; /* work[n][t][u][v] */
    double T = alpha * (X * X + Y * Y + Z * Z);
    for (int n = L; n >= 0; --n) {
        int lim = L - n;
        for (int t = 0; t <= lim; ++t)
            for (int u = 0; u <= lim - t; ++u)
                for (int v = 0; v <= lim - t - u; ++v) {
                    double r;
                    if (t > 0) {
                        r = X * work[n + 1][t - 1][u][v];
                        if (t > 1) r += (t - 1) * work[n + 1][t - 2][u][v];
                    } else if (u > 0) {
                        r = Y * work[n + 1][t][u - 1][v];
                        if (u > 1) r += (u - 1) * work[n + 1][t][u - 2][v];
                    } else if (v > 0) {
                        r = Z * work[n + 1][t][u][v - 1];
                        if (v > 1) r += (v - 1) * work[n + 1][t][u][v - 2];
                    } else {
                        r = pow(-2.0 * alpha, n) * or_boys(n, T);
                    }
                    work[n][t][u][v] = r;
                }
    }
    for (int t = 0; t <= L; ++t)
        for (int u = 0; u <= L - t; ++u)
            for (int v = 0; v <= L - t - u; ++v)
                Rout[(t * RD + u) * RD + v] = work[0][t][u][v];
}

/* Nuclear attraction integrals, Eq. 4, of two primitives to a unit charge at C:
 * <a| 1/|r-C| |b> = (2 pi / p) K_ab sum_tuv E^x_t E^y_u E^z_v R_tuv(p, P-C). */
static double prim_nuclear(or_ws *ws, double a, const double *A, const int *la, double b,
                           const double *B, const int *lb, const double *C)
{
    double p = a + b, mu = a * b / p, r2 = 0.0, P[3];
    double (*E)[EDIM][EDIM][2 * EDIM] = ws->Eab;
    for (int x = 0; x < 3; ++x) {
        P[x] = (a * A[x] + b * B[x]) / p;
        r2 += (A[x] - B[x]) * (A[x] - B[x]);
        hermite_E(la[x], lb[x], P[x] - A[x], P[x] - B[x], 0.5 / p, E[x]);
    }
    int L = la[0] + la[1] + la[2] + lb[0] + lb[1] + lb[2];
    double *R = ws->R;
    hermite_R(ws, L, p, P[0] - C[0], P[1] - C[1], P[2] - C[2], R);
    double s = 0.0;
    for (int t = 0; t <= la[0] + lb[0]; ++t)
        for (int u = 0; u <= la[1] + lb[1]; ++u)
            for (int v = 0; v <= la[2] + lb[2]; ++v)
                s += E[0][la[0]][lb[0]][t] * E[1][la[1]][lb[1]][u] * E[2][la[2]][lb[2]][v] *
                     R[(t * RD + u) * RD + v];
    return 2.0 * OR_PI / p * exp(-mu * r2) * s;
}

/* S, T, V (Eqs. 2-4) for all basis-function pairs, row-major nbf x nbf. */
void or_one_electron(const or_basis *B, double *S, double *T, double *V)
{
    int n = B->nbf;
    or_ws *ws = ws_new();
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            int si = B->bf_shell[i], sj = B->bf_shell[j];
            const double *A = centre(B, si), *Bc = centre(B, sj);
            const int *li = B->bf_lmn + 3 * i, *lj = B->bf_lmn + 3 * j;
            const double *ci = B->bf_coef + B->bf_coef_off[i];
            const double *cj = B->bf_coef + B->bf_coef_off[j];
            double s = 0.0, t = 0.0, v = 0.0;
            for (int k = 0; k < B->sh_nprim[si]; ++k)
                for (int m = 0; m < B->sh_nprim[sj]; ++m) {
                    double a = B->exps[B->sh_prim[si] + k], b = B->exps[B->sh_prim[sj] + m];
                    double w = ci[k] * cj[m];
                    s += w * prim_overlap(a, A, li, b, Bc, lj);
                    t += w * prim_kinetic(a, A, li, b, Bc, lj);
                    for (int at = 0; at < B->natom; ++at)
                        v -= w * B->Z[at] * prim_nuclear(ws, a, A, li, b, Bc, lj, B->xyz + 3 * at);
                }
            if (S) S[i * n + j] = s;
            if (T) T[i * n + j] = t;
            if (V) V[i * n + j] = v;
        }
    free(ws);
}

/* Nuclear repulsion sum_{A<B} Z_A Z_B / R_AB, the constant term of the total
 * energy (Szabo-Ostlund, the textbook the paper's SCF follows). */
double or_nuclear_repulsion(const or_basis *B)
{
    double e = 0.0;
    for (int a = 0; a < B->natom; ++a)
        for (int b = 0; b < a; ++b) {
            double r2 = 0.0;
            for (int x = 0; x < 3; ++x) {
                double d = B->xyz[3 * a + x] - B->xyz[3 * b + x];
                r2 += d * d;
            }
            e += B->Z[a] * B->Z[b] / sqrt(r2);
        }
    return e;
}

/* ------------------------------------------------------------------ */
/* Electron repulsion integrals (Eq. 5), McMurchie-Davidson              */
/* ------------------------------------------------------------------ */

/* Full contracted block (AB|CD) for shells A,B,C,D:
 * out[((i*nb + j)*nc + k)*nd + l] over the Cartesian components.
 * Primitive quartet:
 *   (ab|cd) = 2 pi^{5/2} / (p q sqrt(p+q)) K_ab K_cd
 *             sum_{tuv} E^{ab}_{tuv} sum_{tau nu phi} (-1)^{tau+nu+phi}
 *             E^{cd}_{tau nu phi} R_{t+tau, u+nu, v+phi}(pq/(p+q), P-Q). */
static void eri_block(or_ws *ws, const or_basis *B, int sA, int sB, int sC, int sD, double *out)
{
    int l[4] = {B->sh_l[sA], B->sh_l[sB], B->sh_l[sC], B->sh_l[sD]};
    int sh[4] = {sA, sB, sC, sD};
    int nc[4];
    for (int x = 0; x < 4; ++x) nc[x] = OR_NCART(l[x]);
    int ntot = nc[0] * nc[1] * nc[2] * nc[3];
    for (int x = 0; x < ntot; ++x) out[x] = 0.0;
    const double *A = centre(B, sA), *Bc = centre(B, sB), *C = centre(B, sC), *D = centre(B, sD);
    int L = l[0] + l[1] + l[2] + l[3];
    double (*Eab)[EDIM][EDIM][2 * EDIM] = ws->Eab, (*Ecd)[EDIM][EDIM][2 * EDIM] = ws->Ecd;
    double *R = ws->R;
    int pw[4][OR_MAXCART][3];
    const double *cf[4][OR_MAXCART];
    for (int x = 0; x < 4; ++x)
        for (int c = 0; c < nc[x]; ++c) {
            int bf = B->sh_bf[sh[x]] + c;
            pw[x][c][0] = B->bf_lmn[3 * bf];
            pw[x][c][1] = B->bf_lmn[3 * bf + 1];
            pw[x][c][2] = B->bf_lmn[3 * bf + 2];
            cf[x][c] = B->bf_coef + B->bf_coef_off[bf];
        }
    for (int ka = 0; ka < B->sh_nprim[sA]; ++ka)
        for (int kb = 0; kb < B->sh_nprim[sB]; ++kb) {
            double a = B->exps[B->sh_prim[sA] + ka], b = B->exps[B->sh_prim[sB] + kb];
            double p = a + b, P[3], rab2 = 0.0;
            for (int x = 0; x < 3; ++x) {
                P[x] = (a * A[x] + b * Bc[x]) / p;
                rab2 += (A[x] - Bc[x]) * (A[x] - Bc[x]);
                hermite_E(l[0], l[1], P[x] - A[x], P[x] - Bc[x], 0.5 / p, Eab[x]);
            }
            double Kab = exp(-a * b / p * rab2);
            for (int kc = 0; kc < B->sh_nprim[sC]; ++kc)
                for (int kd = 0; kd < B->sh_nprim[sD]; ++kd) {
                    double c = B->exps[B->sh_prim[sC] + kc], d = B->exps[B->sh_prim[sD] + kd];
                    double q = c + d, Q[3], rcd2 = 0.0;
                    for (int x = 0; x < 3; ++x) {
                        Q[x] = (c * C[x] + d * D[x]) / q;
                        rcd2 += (C[x] - D[x]) * (C[x] - D[x]);
                        hermite_E(l[2], l[3], Q[x] - C[x], Q[x] - D[x], 0.5 / q, Ecd[x]);
                    }
                    double Kcd = exp(-c * d / q * rcd2);
                    double alpha = p * q / (p + q);
                    hermite_R(ws, L, alpha, P[0] - Q[0], P[1] - Q[1], P[2] - Q[2], R);
                    double pref = 2.0 * pow(OR_PI, 2.5) / (p * q * sqrt(p + q)) * Kab * Kcd;
                    int o = 0;
                    for (int i = 0; i < nc[0]; ++i)
                        for (int j = 0; j < nc[1]; ++j)
                            for (int k = 0; k < nc[2]; ++k)
                                for (int m = 0; m < nc[3]; ++m, ++o) {
                                    const int *pi = pw[0][i], *pj = pw[1][j], *pk = pw[2][k], *pm = pw[3][m];
                                    double s = 0.0;
                                    for (int t = 0; t <= pi[0] + pj[0]; ++t)
                                        for (int u = 0; u <= pi[1] + pj[1]; ++u)
                                            for (int v = 0; v <= pi[2] + pj[2]; ++v) {
                                                double eb = Eab[0][pi[0]][pj[0]][t] *
                                                            Eab[1][pi[1]][pj[1]][u] *
                                                            Eab[2][pi[2]][pj[2]][v];
                                                if (eb == 0.0) continue;
                                                double sk = 0.0;
                                                for (int tt = 0; tt <= pk[0] + pm[0]; ++tt)
                                                    for (int uu = 0; uu <= pk[1] + pm[1]; ++uu)
                                                        for (int vv = 0; vv <= pk[2] + pm[2]; ++vv) {
                                                            double ek = Ecd[0][pk[0]][pm[0]][tt] *
                                                                        Ecd[1][pk[1]][pm[1]][uu] *
                                                                        Ecd[2][pk[2]][pm[2]][vv];
                                                            double sg = ((tt + uu + vv) % 2) ? -1.0 : 1.0;
                                                            sk += sg * ek *
                                                                  R[((t + tt) * RD + (u + uu)) * RD + (v + vv)];
                                                        }
                                                s += eb * sk;
                                            }
                                    double w = cf[0][i][ka] * cf[1][j][kb] * cf[2][k][kc] * cf[3][m][kd];
                                    out[o] += w * pref * s;
                                }
                }
        }
}

static int max_block(const or_basis *B)
{
    int lm = 0;
    for (int s = 0; s < B->nshell; ++s)
        if (B->sh_l[s] > lm) lm = B->sh_l[s];
    int n = OR_NCART(lm);
    return n * n * n * n;
}

/* One contracted integral (ij|kl) over basis functions. */
double or_eri(const or_basis *B, int i, int j, int k, int l)
{
    int s[4] = {B->bf_shell[i], B->bf_shell[j], B->bf_shell[k], B->bf_shell[l]};
    double *blk = (double *)malloc(sizeof(double) * max_block(B));
    or_ws *ws = ws_new();
    eri_block(ws, B, s[0], s[1], s[2], s[3], blk);
    int nj = OR_NCART(B->sh_l[s[1]]), nk = OR_NCART(B->sh_l[s[2]]), nl = OR_NCART(B->sh_l[s[3]]);
    int ii = i - B->sh_bf[s[0]], jj = j - B->sh_bf[s[1]], kk = k - B->sh_bf[s[2]], ll = l - B->sh_bf[s[3]];
    double v = blk[((ii * nj + jj) * nk + kk) * nl + ll];
    free(blk); free(ws);
    return v;
}

/* The contracted block for four shells, written row-major as in eri_block. */
void or_eri_shell_block(const or_basis *B, int sA, int sB, int sC, int sD, double *out)
{
    or_ws *ws = ws_new();
    eri_block(ws, B, sA, sB, sC, sD, out);
    free(ws);
}

/* Schwarz factors (not in the paper: the screening rule is a reading of it).
 * Q_AB = sqrt(max_{a in A, b in B} |(ab|ab)|) for all shell pairs,
 * nshell x nshell row-major (symmetric); the shell loop is split over the
 * OpenMP threads (each writes its own entries). */
void or_schwarz(const or_basis *B, double *Q)
{
    int ns = B->nshell;
#ifdef _OPENMP
#pragma omp parallel
#endif
    {
    double *blk = (double *)malloc(sizeof(double) * max_block(B)); or_ws *ws = ws_new();
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
    for (int a = 0; a < ns; ++a)
        for (int b = 0; b <= a; ++b) {
            eri_block(ws, B, a, b, a, b, blk);
            int na = OR_NCART(B->sh_l[a]), nb = OR_NCART(B->sh_l[b]);
            double m = 0.0;
            for (int i = 0; i < na; ++i)
                for (int j = 0; j < nb; ++j) {
                    double v = fabs(blk[((i * nb + j) * na + i) * nb + j]);
                    if (v > m) m = v;
                }
            Q[a * ns + b] = Q[b * ns + a] = sqrt(m);
        }
    free(blk); free(ws);
    }
}

/* All N^4 integrals of Eq. 5 (small N only), row-major [i][j][k][l]. */
void or_eri_tensor(const or_basis *B, double *G)
{
    int n = B->nbf, ns = B->nshell;
    double *blk = (double *)malloc(sizeof(double) * max_block(B)); or_ws *ws = ws_new();
    for (int a = 0; a < ns; ++a)
        for (int b = 0; b < ns; ++b)
            for (int c = 0; c < ns; ++c)
                for (int d = 0; d < ns; ++d) {
                    eri_block(ws, B, a, b, c, d, blk);
                    int na = OR_NCART(B->sh_l[a]), nb = OR_NCART(B->sh_l[b]);
                    int nc = OR_NCART(B->sh_l[c]), nd = OR_NCART(B->sh_l[d]);
                    int o = 0;
                    for (int i = 0; i < na; ++i)
                        for (int j = 0; j < nb; ++j)
                            for (int k = 0; k < nc; ++k)
                                for (int l = 0; l < nd; ++l, ++o) {
                                    long I = B->sh_bf[a] + i, J = B->sh_bf[b] + j;
                                    long K = B->sh_bf[c] + k, L = B->sh_bf[d] + l;
                                    G[((I * n + J) * n + K) * n + L] = blk[o];
                                }
                }
    free(blk); free(ws);
}

/* Add one unique integral v = (ij|kl) to J and K through every distinct
 * index permutation that the 8-fold symmetry of Eq. 5 maps it to:
 * J_ab += (ab|cd) P_cd and K_ad += (ab|cd) P_bc for each distinct (a,b,c,d). */
static void digest(int i, int j, int k, int l, double v, const double *P, double *J,
                   double *K, int n)
{
    int perm[8][4] = {{i, j, k, l}, {j, i, k, l}, {i, j, l, k}, {j, i, l, k},
                      {k, l, i, j}, {l, k, i, j}, {k, l, j, i}, {l, k, j, i}};
    for (int p = 0; p < 8; ++p) {
        int dup = 0;
        for (int q = 0; q < p && !dup; ++q)
            dup = perm[q][0] == perm[p][0] && perm[q][1] == perm[p][1] &&
                  perm[q][2] == perm[p][2] && perm[q][3] == perm[p][3];
        if (dup) continue;
        int a = perm[p][0], b = perm[p][1], c = perm[p][2], d = perm[p][3];
        J[a * n + b] += v * P[c * n + d];
        K[a * n + d] += v * P[b * n + c];
    }
}

/* Inside a unique shell quartet (A>=B, C>=D, AB>=CD) the block still holds
 * several members of one symmetry orbit when shells coincide.  Returns
 * nonzero for the members to SKIP, keeping exactly one per orbit: i>=j when
 * A==B, k>=l when C==D, and pair(ij)>=pair(kl) when (A,B)==(C,D). */
static int unique_in_block(int A, int B, int C, int D, int i, int j, int k, int l)
{
    if (A == B && j > i) return 1;
    if (C == D && l > k) return 1;
    if (A == C && B == D) {
        long ij = (long)i * (i + 1) / 2 + j, kl = (long)k * (k + 1) / 2 + l;
        if (i < j) ij = (long)j * (j + 1) / 2 + i;
        if (k < l) kl = (long)l * (l + 1) / 2 + k;
        if (kl > ij) return 1;
    }
    return 0;
}

/* J and K of the J/K equation (Sec. "Technical details") for a density P
 * (nbf x nbf, row-major), over the unique shell quartets A>=B, C>=D,
 * (AB)>=(CD), each integral then expanded through
 * digest().  tau > 0 enables the Schwarz rule with the oracle's own Q.
 * nthreads > 1 splits the outer shell loop over OpenMP threads, each with
 * private J, K that are summed at the end.  Returns the number of shell
 * quartets evaluated. */
long or_jk(const or_basis *B, const double *P, double *J, double *K, double tau, int nthreads)
{
    int n = B->nbf, ns = B->nshell;
    double *Q = NULL;
    if (tau > 0.0) {
        Q = (double *)malloc(sizeof(double) * ns * ns);
        or_schwarz(B, Q);
    }
    memset(J, 0, sizeof(double) * n * n);
    memset(K, 0, sizeof(double) * n * n);
    long count = 0;
    if (nthreads < 1) nthreads = 1;
#ifdef _OPENMP
#pragma omp parallel num_threads(nthreads) reduction(+ : count)
#endif
    {
        double *Jt = (double *)calloc((size_t)n * n, sizeof(double));
        double *Kt = (double *)calloc((size_t)n * n, sizeof(double));
        double *blk = (double *)malloc(sizeof(double) * max_block(B)); or_ws *ws = ws_new();
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int A = 0; A < ns; ++A)
            for (int Bs = 0; Bs <= A; ++Bs)
                for (int C = 0; C <= A; ++C)
                    for (int D = 0; D <= (C == A ? Bs : C); ++D) {
                        if (Q && Q[A * ns + Bs] * Q[C * ns + D] < tau) continue;
                        ++count;
                        eri_block(ws, B, A, Bs, C, D, blk);
                        int na = OR_NCART(B->sh_l[A]), nb = OR_NCART(B->sh_l[Bs]);
                        int nc = OR_NCART(B->sh_l[C]), nd = OR_NCART(B->sh_l[D]);
                        int o = 0;
                        for (int i = 0; i < na; ++i)
                            for (int j = 0; j < nb; ++j)
                                for (int k = 0; k < nc; ++k)
                                    for (int l = 0; l < nd; ++l, ++o) {
                                        int I = B->sh_bf[A] + i, Jb = B->sh_bf[Bs] + j;
                                        int Kb = B->sh_bf[C] + k, L = B->sh_bf[D] + l;
                                        if (unique_in_block(A, Bs, C, D, I, Jb, Kb, L)) continue;
                                        digest(I, Jb, Kb, L, blk[o], P, Jt, Kt, n);
                                    }
                    }
        free(blk); free(ws);
#ifdef _OPENMP
#pragma omp critical
#endif
        {
            for (long x = 0; x < (long)n * n; ++x) {
                J[x] += Jt[x];
                K[x] += Kt[x];
            }
        }
        free(Jt);
        free(Kt);
    }
    free(Q);
    return count;
}

/* Rows of J and K straight from the definitions:
 * J_ij = sum_kl (ij|kl) P_kl and K_il = sum_jk (ij|kl) P_jk for each i in
 * rows[0..nrows), all j (resp. l).  Jrows/Krows are nrows x nbf.  Every
 * shell quartet (I J|K L) with I the shell of row i is evaluated (no
 * permutational symmetry), except those whose terms are all zero because
 * both density blocks they meet, P[K,L] and P[J,K], are zero; tau > 0
 * applies the Schwarz rule. */
void or_jk_rows(const or_basis *B, const double *P, int nrows, const int *rows,
                double *Jrows, double *Krows, double tau, int nthreads)
{
    int n = B->nbf, ns = B->nshell;
    double *Q = NULL;
    if (tau > 0.0) {
        Q = (double *)malloc(sizeof(double) * ns * ns);
        or_schwarz(B, Q);
    }
    /* nz[X*ns+Y]: the density block of shells X, Y has a nonzero entry */
    char *nz = (char *)calloc((size_t)ns * ns, 1);
    for (int X = 0; X < ns; ++X)
        for (int Y = 0; Y < ns; ++Y)
            for (int x = B->sh_bf[X]; x < B->sh_bf[X + 1] && !nz[X * ns + Y]; ++x)
                for (int y = B->sh_bf[Y]; y < B->sh_bf[Y + 1]; ++y)
                    if (P[x * n + y] != 0.0) { nz[X * ns + Y] = 1; break; }
    memset(Jrows, 0, sizeof(double) * nrows * n);
    memset(Krows, 0, sizeof(double) * nrows * n);
    if (nthreads < 1) nthreads = 1;
    for (int r = 0; r < nrows; ++r) {
        int i = rows[r], I = B->bf_shell[i], ii = i - B->sh_bf[I];
#ifdef _OPENMP
#pragma omp parallel num_threads(nthreads)
#endif
        {
            double *Jt = (double *)calloc(n, sizeof(double));
            double *Kt = (double *)calloc(n, sizeof(double));
            double *blk = (double *)malloc(sizeof(double) * max_block(B)); or_ws *ws = ws_new();
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
            for (int Js = 0; Js < ns; ++Js)
                for (int Ks = 0; Ks < ns; ++Ks)
                    for (int Ls = 0; Ls < ns; ++Ls) {
                        if (!nz[Ks * ns + Ls] && !nz[Js * ns + Ks]) continue;
                        if (Q && Q[I * ns + Js] * Q[Ks * ns + Ls] < tau) continue;
                        eri_block(ws, B, I, Js, Ks, Ls, blk);
                        int nb = OR_NCART(B->sh_l[Js]), nc = OR_NCART(B->sh_l[Ks]), nd = OR_NCART(B->sh_l[Ls]);
                        for (int j = 0; j < nb; ++j)
                            for (int k = 0; k < nc; ++k)
                                for (int l = 0; l < nd; ++l) {
                                    double v = blk[((ii * nb + j) * nc + k) * nd + l];
                                    int jb = B->sh_bf[Js] + j, kb = B->sh_bf[Ks] + k, lb = B->sh_bf[Ls] + l;
                                    Jt[jb] += v * P[kb * n + lb];
                                    Kt[lb] += v * P[jb * n + kb];
                                }
                    }
            free(blk); free(ws);
#ifdef _OPENMP
#pragma omp critical
#endif
            {
                for (int x = 0; x < n; ++x) {
                    Jrows[r * n + x] += Jt[x];
                    Krows[r * n + x] += Kt[x];
                }
            }
            free(Jt);
            free(Kt);
        }
    }
    free(nz);
    free(Q);
}

/* Number of shell quartets that or_jk evaluates: unique, and surviving
 * the Schwarz rule when tau > 0. */
long or_count_quartets(const or_basis *B, double tau)
{
    int ns = B->nshell;
    double *Q = NULL;
    if (tau > 0.0) {
        Q = (double *)malloc(sizeof(double) * ns * ns);
        or_schwarz(B, Q);
    }
    long count = 0;
    for (int A = 0; A < ns; ++A)
        for (int Bs = 0; Bs <= A; ++Bs)
            for (int C = 0; C <= A; ++C)
                for (int D = 0; D <= (C == A ? Bs : C); ++D) {
                    if (Q && Q[A * ns + Bs] * Q[C * ns + D] < tau) continue;
                    ++count;
                }
    free(Q);
    return count;
}

/* Evaluate and digest an explicit list of unique shell quartets
 * (quads: nq x 4 shell indices, each with A>=B, C>=D, AB>=CD).  Used to
 * time the oracle on a bounded sample of a large workload.  J, K are
 * accumulated (not cleared). */
void or_jk_quartets(const or_basis *B, const double *P, long nq, const int *quads,
                    double *J, double *K)
{
    int n = B->nbf;
    double *blk = (double *)malloc(sizeof(double) * max_block(B)); or_ws *ws = ws_new();
    for (long q = 0; q < nq; ++q) {
        int A = quads[4 * q], Bs = quads[4 * q + 1], C = quads[4 * q + 2], D = quads[4 * q + 3];
        eri_block(ws, B, A, Bs, C, D, blk);
        int na = OR_NCART(B->sh_l[A]), nb = OR_NCART(B->sh_l[Bs]);
        int nc = OR_NCART(B->sh_l[C]), nd = OR_NCART(B->sh_l[D]);
        int o = 0;
        for (int i = 0; i < na; ++i)
            for (int j = 0; j < nb; ++j)
                for (int k = 0; k < nc; ++k)
                    for (int l = 0; l < nd; ++l, ++o) {
                        int I = B->sh_bf[A] + i, Jb = B->sh_bf[Bs] + j;
                        int Kb = B->sh_bf[C] + k, L = B->sh_bf[D] + l;
                        if (unique_in_block(A, Bs, C, D, I, Jb, Kb, L)) continue;
                        digest(I, Jb, Kb, L, blk[o], P, J, K, n);
                    }
    }
    free(blk); free(ws);
}

int or_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
