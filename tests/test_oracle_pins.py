"""Pins of the CPU oracle against things other than itself.

* Boys function: F_m(0), the erf closed form of F_0, the large-T asymptote,
  the downward recursion and direct Gauss-Legendre quadrature.
* The Szabo-Ostlund H2 / STO-3G worked example (printed to 4 decimals).
* The closed-form (ss|ss) integral with F_0(T) = sqrt(pi/T) erf(sqrt T) / 2.
* The single-Gaussian He atom, E(a) = 3a - 8 sqrt(2a/pi) + 2 sqrt(a/pi).
* Brute-force quadrature (tests/quadrature.py) of S, T, V and ERIs over
  s, p, d shells (and f, g for the oracle's own range), which uses no Boys
  function and no recurrence.
* Invariants: 8-fold symmetry, Schwarz inequality, positive semidefinite
  ERI supermatrix, symmetric J/K, rotation / translation / permutation
  invariance of the energy, idempotency at convergence.
* J/K from the unique-quartet digestion against the plain contraction of
  the full tensor (a different code path in the oracle).
* DIIS: the exact root of an affine error map, a null-space least-squares
  solve of the same constrained minimum; Loewdin: X S X = I.
* UHF: one-electron closed form and core eigenvalue, UHF = RHF for closed
  shells, spin-swap symmetry and the <S^2> >= S_z(S_z+1) bound.
* MP2: minimal-basis H2 closed form, the spin-orbital antisymmetrised form,
  size consistency with the R^-3 dipole tail.
* Nuclear gradient: sympy's exact derivative of the closed-form H2 energy
  (one s Gaussian per atom); zero net force and torque.
* The stored rows of the 150-atom molecule: made for the current input and
  symmetric where two stored rows cross.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from synth import h_line, lattice_molecule, random_shells_molecule
from synth.molecules import _pack
from quadrature import QuadBasis

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- Boys

@pytest.mark.parametrize("m", range(0, 13))
def test_boys_at_zero(m):
    assert oracle.boys(m, 0.0) == pytest.approx(1.0 / (2 * m + 1), rel=1e-15)


@pytest.mark.parametrize("T", [1e-8, 1e-3, 0.1, 0.7, 2.0, 5.5, 11.0, 17.3, 29.99, 30.0, 30.01, 45.0, 120.0])
def test_boys_f0_erf_closed_form(T):
    ref = 0.5 * math.sqrt(math.pi / T) * math.erf(math.sqrt(T))
    assert oracle.boys(0, T) == pytest.approx(ref, rel=2e-15, abs=1e-300)


@pytest.mark.parametrize("m", [0, 1, 3, 6, 8, 12])
@pytest.mark.parametrize("T", [60.0, 100.0, 400.0])
def test_boys_large_T_asymptote(m, T):
    # F_m(T) ~ (2m-1)!! / 2^{m+1} sqrt(pi / T^{2m+1}) up to O(e^{-T}).
    df = 1.0
    for k in range(2 * m - 1, 0, -2):
        df *= k
    ref = df / 2 ** (m + 1) * math.sqrt(math.pi / T ** (2 * m + 1))
    assert oracle.boys(m, T) == pytest.approx(ref, rel=1e-14)


@pytest.mark.parametrize("T", [0.05, 1.0, 7.0, 20.0, 29.0, 31.0, 50.0])
def test_boys_downward_recursion(T):
    # F_m = (2T F_{m+1} + e^{-T}) / (2m+1)
    for m in range(0, 12):
        lhs = oracle.boys(m, T)
        rhs = (2 * T * oracle.boys(m + 1, T) + math.exp(-T)) / (2 * m + 1)
        assert lhs == pytest.approx(rhs, rel=5e-15)


@pytest.mark.parametrize("m", [0, 2, 5, 9])
@pytest.mark.parametrize("T", [0.0, 0.3, 4.0, 15.0, 33.0])
def test_boys_gauss_legendre(m, T):
    x, w = np.polynomial.legendre.leggauss(300)
    t = 0.5 * (x + 1.0)
    ref = 0.5 * np.sum(w * t ** (2 * m) * np.exp(-T * t * t))
    assert oracle.boys(m, T) == pytest.approx(ref, rel=1e-13)


# ---------------------------------------------------------------- Szabo-Ostlund H2

def _h2(z2=1):
    g = json.load(open(os.path.join(GOLDEN, "h2_sto3g.json")))
    a, d = g["exponents"], g["coefficients"]
    m = _pack([1, z2], [[0, 0, 0], [g["R_bohr"], 0, 0]], [(0, 0, a, d), (1, 0, a, d)], "h2", 0,
              n_electrons=2)
    return m, g


def test_szabo_ostlund_h2_sto3g():
    m, g = _h2()
    pr, tol = g["printed"], g["tolerance"]
    B = oracle.Basis(m)
    S, T, V = B.one_electron()
    assert S[0, 1] == pytest.approx(pr["S12"], abs=tol)
    assert T[0, 0] == pytest.approx(pr["T11"], abs=tol)
    assert T[0, 1] == pytest.approx(pr["T12"], abs=tol)
    H = T + V
    assert H[0, 0] == pytest.approx(pr["H11"], abs=tol)
    assert H[0, 1] == pytest.approx(pr["H12"], abs=tol)
    # nucleus-1 attraction alone: give atom 2 zero charge
    m1, _ = _h2(z2=0)
    _, _, V1 = oracle.Basis(m1).one_electron()
    assert V1[0, 0] == pytest.approx(pr["V1_11"], abs=tol)
    assert V1[0, 1] == pytest.approx(pr["V1_12"], abs=tol)
    assert V1[1, 1] == pytest.approx(pr["V1_22"], abs=tol)
    assert B.eri(0, 0, 0, 0) == pytest.approx(pr["eri_11_11"], abs=tol)
    assert B.eri(0, 0, 1, 1) == pytest.approx(pr["eri_11_22"], abs=tol)
    assert B.eri(1, 0, 0, 0) == pytest.approx(pr["eri_21_11"], abs=tol)
    assert B.eri(1, 0, 1, 0) == pytest.approx(pr["eri_21_21"], abs=tol)
    r = oracle.rhf(m, max_iter=50, e_tol=1e-12)
    assert r.converged
    assert r.eps[0] == pytest.approx(pr["eps1"], abs=tol)
    assert r.eps[1] == pytest.approx(pr["eps2"], abs=tol)
    assert r.e_elec == pytest.approx(pr["E_elec"], abs=tol)
    assert r.energy == pytest.approx(pr["E_tot"], abs=tol)


# ---------------------------------------------------------------- closed forms

def _norm_s(a):
    return (2.0 * a / math.pi) ** 0.75


def _closed_ssss(mol, i, j, k, l):
    """Contracted (ss|ss) from the closed form, normalised independently."""
    def shell(s):
        p0, K = mol.shell_prim[s], mol.shell_nprim[s]
        e = mol.exps[p0:p0 + K]
        c = mol.coefs[p0:p0 + K] * np.array([_norm_s(x) for x in e])
        n2 = sum(c[u] * c[v] * (math.pi / (e[u] + e[v])) ** 1.5 for u in range(K) for v in range(K))
        return e, c / math.sqrt(n2), mol.xyz[mol.shell_atom[s]]
    (ea, ca, A), (eb, cb, B), (ec, cc, C), (ed, cd, D) = [shell(s) for s in (i, j, k, l)]
    tot = 0.0
    for a, wa in zip(ea, ca):
        for b, wb in zip(eb, cb):
            p = a + b
            P = (a * A + b * B) / p
            kab = math.exp(-a * b / p * np.sum((A - B) ** 2))
            for c, wc in zip(ec, cc):
                for d, wd in zip(ed, cd):
                    q = c + d
                    Q = (c * C + d * D) / q
                    kcd = math.exp(-c * d / q * np.sum((C - D) ** 2))
                    T = p * q / (p + q) * np.sum((P - Q) ** 2)
                    f0 = 1.0 if T < 1e-15 else 0.5 * math.sqrt(math.pi / T) * math.erf(math.sqrt(T))
                    tot += wa * wb * wc * wd * 2 * math.pi ** 2.5 / (p * q * math.sqrt(p + q)) * kab * kcd * f0
    return tot


def test_ssss_closed_form_h_line():
    mol = h_line()
    B = oracle.Basis(mol)
    rng = np.random.default_rng(5)
    for _ in range(40):
        i, j, k, l = rng.integers(0, mol.nshell, size=4)
        assert B.eri(i, j, k, l) == pytest.approx(_closed_ssss(mol, i, j, k, l), rel=1e-13, abs=1e-15)


@pytest.mark.parametrize("alpha", [0.3, 0.7671, 2.5])
def test_single_gaussian_helium(alpha):
    m = _pack([2], [[0.1, -0.2, 0.3]], [(0, 0, [alpha], [1.0])], "he", 0, n_electrons=2)
    r = oracle.rhf(m, max_iter=5, e_tol=1e-13)
    ref = 3 * alpha - 8 * math.sqrt(2 * alpha / math.pi) + 2 * math.sqrt(alpha / math.pi)
    assert r.energy == pytest.approx(ref, rel=1e-13)
    # minimum over alpha: E = -(8 sqrt 2 - 2)^2 / (12 pi) ~ -2.3010
    if alpha == 0.7671:
        assert r.energy == pytest.approx(-(8 * math.sqrt(2) - 2) ** 2 / (12 * math.pi), abs=2e-6)


# ---------------------------------------------------------------- quadrature

# f and g shells (l = 3, 4) are beyond the GPU path (l <= 2) but inside the
# oracle's range: pinned here for the f/g row that comes next
@pytest.mark.parametrize("ls,seed", [((0, 1, 2), 3), ((2, 2, 1), 11), ((1, 0), 4), ((3, 1), 5), ((4, 2), 6)])
def test_one_electron_vs_quadrature(ls, seed):
    mol = random_shells_molecule(ls, seed, nprim=(1, 2), Z=np.array([1, 3, 2][:len(ls)], dtype=np.int32))
    B = oracle.Basis(mol)
    S, T, V = B.one_electron()
    Q = QuadBasis(mol)
    n = B.nbf
    for i in range(n):
        assert S[i, i] == pytest.approx(1.0, abs=1e-13)
        for j in range(n):
            assert S[i, j] == pytest.approx(Q.overlap(i, j), abs=1e-12)
            assert T[i, j] == pytest.approx(Q.kinetic(i, j), abs=1e-11)
    rng = np.random.default_rng(seed)
    for _ in range(12):
        i, j = rng.integers(0, n, size=2)
        assert V[i, j] == pytest.approx(Q.nuclear(i, j), abs=1e-10)


@pytest.mark.parametrize("ls,seed", [((1, 0, 1, 0), 1), ((1, 1, 1, 1), 2), ((2, 0, 1, 0), 3),
                                     ((2, 1, 2, 0), 4), ((2, 2, 2, 2), 5), ((0, 0, 0, 0), 6),
                                     ((3, 0, 1, 0), 7), ((3, 2, 3, 1), 8), ((4, 0, 2, 0), 9)])
def test_eri_vs_quadrature(ls, seed):
    mol = random_shells_molecule(ls, seed, nprim=(1, 2), exp_range=(0.3, 2.5))
    B = oracle.Basis(mol)
    Q = QuadBasis(mol)
    sb = B.shell_bf
    blk = B.eri_shell_block(0, 1, 2, 3)
    rng = np.random.default_rng(seed)
    idx = [tuple(rng.integers(0, blk.shape[x]) for x in range(4)) for _ in range(10)]
    for (a, b, c, d) in idx:
        ref = Q.eri(sb[0] + a, sb[1] + b, sb[2] + c, sb[3] + d)
        assert blk[a, b, c, d] == pytest.approx(ref, rel=1e-9, abs=1e-12)


# ---------------------------------------------------------------- invariants

def _small_spd(seed=7):
    return random_shells_molecule((2, 1, 0, 1, 2), seed, nprim=(1, 2), exp_range=(0.2, 3.0), box=3.0,
                                  Z=np.array([6, 1, 1, 8, 1], dtype=np.int32))


def test_eri_tensor_symmetry_schwarz_psd():
    mol = _small_spd()
    B = oracle.Basis(mol)
    G = B.eri_tensor()
    for perm in [(1, 0, 2, 3), (0, 1, 3, 2), (2, 3, 0, 1), (3, 2, 1, 0)]:
        np.testing.assert_allclose(G, G.transpose(perm), atol=1e-13, rtol=0)
    n = B.nbf
    diag = np.einsum("ijij->ij", G)
    bound = np.sqrt(np.einsum("ij,kl->ijkl", diag, diag))
    assert np.all(np.abs(G) <= bound * (1 + 1e-12) + 1e-14)
    M = G.reshape(n * n, n * n)
    assert np.linalg.eigvalsh(0.5 * (M + M.T)).min() > -1e-12
    Q = B.schwarz()
    sb = B.shell_bf
    for a in range(mol.nshell):
        for b in range(mol.nshell):
            blk = diag[sb[a]:sb[a + 1], sb[b]:sb[b + 1]]
            assert Q[a, b] == pytest.approx(math.sqrt(np.abs(blk).max()), rel=1e-14)


def _rand_density(n, seed, nocc=None):
    rng = np.random.default_rng(seed)
    C = rng.normal(size=(n, nocc or max(1, n // 3))) / math.sqrt(n)
    return C @ C.T


def test_jk_digest_matches_full_contraction():
    mol = _small_spd()
    B = oracle.Basis(mol)
    G = B.eri_tensor()
    D = _rand_density(B.nbf, 3)
    J, K, nq = B.jk(D)
    np.testing.assert_allclose(J, np.einsum("ijkl,kl->ij", G, D), atol=1e-12, rtol=0)
    np.testing.assert_allclose(K, np.einsum("ijkl,jk->il", G, D), atol=1e-12, rtol=0)
    ns = mol.nshell
    npair = ns * (ns + 1) // 2
    assert nq == npair * (npair + 1) // 2
    np.testing.assert_allclose(J, J.T, atol=1e-13)
    np.testing.assert_allclose(K, K.T, atol=1e-13)
    assert np.sum(D * J) >= 0 and np.sum(D * K) >= 0
    rows = np.array([0, 4, B.nbf - 1])
    Jr, Kr = B.jk_rows(D, rows)
    np.testing.assert_allclose(Jr, J[rows], atol=1e-12, rtol=0)
    np.testing.assert_allclose(Kr, K[rows], atol=1e-12, rtol=0)
    J2, K2, _ = B.jk(D, nthreads=3)
    np.testing.assert_allclose(J2, J, atol=1e-13)
    np.testing.assert_allclose(K2, K, atol=1e-13)


def test_schwarz_screening_is_bounded():
    mol = lattice_molecule(6, 3, "sp")
    B = oracle.Basis(mol)
    D = _rand_density(B.nbf, 4)
    J0, K0, n0 = B.jk(D)
    tau = 1e-6
    J1, K1, n1 = B.jk(D, tau=tau)
    assert n1 < n0
    assert n1 == B.count_quartets(tau)
    # each dropped integral is below tau in magnitude; each is used in at most
    # 8 places of J and K with |D| entries
    dropped = n0 - n1
    bound = 8 * dropped * 36 * tau * np.abs(D).max()
    assert np.abs(J1 - J0).max() <= bound
    assert np.abs(K1 - K0).max() <= bound


def _rotation(seed):
    rng = np.random.default_rng(seed)
    q, r = np.linalg.qr(rng.normal(size=(3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] *= -1
    return q


def test_energy_invariances():
    mol = random_shells_molecule((1, 0, 2, 1), 21, nprim=(1, 2), exp_range=(0.3, 3.0), box=3.5,
                                 Z=np.array([3, 1, 2, 2], dtype=np.int32))
    e0 = oracle.rhf(mol, max_iter=80, e_tol=1e-11, diis_size=6)
    assert e0.converged
    R = _rotation(1)
    m2 = mol.copy()
    m2.xyz = mol.xyz @ R.T + np.array([0.3, -1.2, 2.0])
    e1 = oracle.rhf(m2, max_iter=80, e_tol=1e-11, diis_size=6)
    assert e1.energy == pytest.approx(e0.energy, abs=1e-9)
    # permute atoms (shells follow their atoms)
    perm = np.array([2, 0, 3, 1])
    inv = np.argsort(perm)
    m3 = mol.copy()
    m3.Z = mol.Z[perm]
    m3.xyz = mol.xyz[perm]
    m3.shell_atom = inv[mol.shell_atom].astype(np.int32)
    e2 = oracle.rhf(m3, max_iter=80, e_tol=1e-11, diis_size=6)
    assert e2.energy == pytest.approx(e0.energy, abs=1e-9)
    # stationarity and idempotency at convergence
    D, S, F = e0.D, e0.S, e0.F
    np.testing.assert_allclose(D @ S @ D, D, atol=1e-6)
    assert np.trace(D @ S) == pytest.approx(mol.n_electrons // 2, abs=1e-9)
    assert np.abs(F @ D @ S - S @ D @ F).max() < 1e-4


def test_scf_h_line_no_diis():
    mol = h_line()
    r = oracle.rhf(mol, max_iter=30, e_tol=1e-8, diis_size=0)
    assert r.converged
    assert r.energy < 0
    # variational: the SCF energy is not above the core-guess energy of D_1
    assert r.energy <= r.energies[0] + 1e-12


def test_jk_rows_with_zero_density_blocks():
    # rows skip quartets whose density blocks are zero: same result as the full build
    mol = _small_spd(9)
    B = oracle.Basis(mol)
    D = _rand_density(B.nbf, 8)
    keep = np.zeros(B.nbf, dtype=bool)
    for s in (0, 3):
        keep[B.shell_bf[s]:B.shell_bf[s + 1]] = True
    D = D * np.outer(keep, keep)
    J, K, _ = B.jk(D)
    rows = np.arange(B.nbf)
    Jr, Kr = B.jk_rows(D, rows)
    np.testing.assert_allclose(Jr, J, atol=1e-13, rtol=0)
    np.testing.assert_allclose(Kr, K, atol=1e-13, rtol=0)


def test_stored_c3_rows_are_consistent():
    """The stored oracle rows of the 150-atom s+p+d molecule were made for
    the density the synthetic generator draws now, and they obey the
    symmetry J_ij = J_ji, K_ij = K_ji wherever two stored rows cross."""
    from synth import shell_supported_density
    gold = np.load(os.path.join(os.path.dirname(__file__), "golden", "c3_rows.npz"))
    mol = lattice_molecule(150, 2, "spd")
    _, shells, rows = shell_supported_density(mol, seed=11)
    assert gold["rows"].tolist() == rows.tolist() and gold["shells"].tolist() == list(shells)
    for M in (gold["J"], gold["K"]):
        sub = M[:, rows]
        assert np.abs(sub - sub.T).max() <= 1e-13 * max(1.0, np.abs(M).max())


def test_diis_recovers_the_root_of_an_affine_error():
    """Pulay's extrapolation (DIIS, named in the paper's SCF description)
    minimises |sum_i c_i e_i| subject to sum_i c_i = 1.  When the error is an
    affine function of F, e(F) = P (F - F*) Q with P, Q invertible, and the
    stored F_i affinely span the space, that minimum is e = 0 at
    sum_i c_i F_i = F*: the extrapolation must return F* itself.  A wrong
    sign, a transposed B matrix or a dropped constraint row fails this."""
    from oracle.scf import diis_extrapolate
    rng = np.random.default_rng(5)
    n = 2
    Fstar = rng.normal(size=(n, n))
    P = rng.normal(size=(n, n)) + 3 * np.eye(n)
    Q = rng.normal(size=(n, n)) + 3 * np.eye(n)
    Fs = [Fstar + rng.normal(size=(n, n)) for _ in range(n * n + 1)]
    es = [P @ (F - Fstar) @ Q for F in Fs]
    assert np.abs(diis_extrapolate(Fs, es) - Fstar).max() < 1e-10
    # with fewer vectors than the space needs, the result is the affine
    # combination whose error is smallest: check it against a brute-force
    # least-squares solve of the same constrained problem
    Fs3, es3 = Fs[:3], es[:3]
    E = np.stack([e.ravel() for e in es3], axis=1)           # columns e_i
    # c = c0 + N t with sum c = 1: c0 = (1,0,0), N spans sum-zero vectors
    N = np.array([[-1.0, -1.0], [1.0, 0.0], [0.0, 1.0]])
    t, *_ = np.linalg.lstsq(E @ N, -E[:, 0], rcond=None)
    c = np.array([1.0, 0.0, 0.0]) + N @ t
    expect = sum(ci * F for ci, F in zip(c, Fs3))
    assert np.abs(diis_extrapolate(Fs3, es3) - expect).max() < 1e-10


def test_diis_drops_vectors_that_make_b_singular():
    """Identical error vectors make the DIIS matrix singular; the oldest is
    dropped until it is not, and one vector alone is returned unchanged."""
    from oracle.scf import diis_extrapolate
    F1, F2 = np.eye(2), 2 * np.eye(2)
    e = np.array([[0.0, 1.0], [-1.0, 0.0]])
    assert np.array_equal(diis_extrapolate([F1, F2], [e, e]), F2)


def test_lowdin_is_the_symmetric_inverse_square_root():
    """X = S^(-1/2) (Loewdin): X symmetric, X S X = I and X X = S^(-1);
    near-singular S raises LinearDependence."""
    from oracle.scf import LinearDependence, lowdin
    mol = lattice_molecule(3, 3, "spd")
    S, _, _ = oracle.Basis(mol).one_electron()
    X = lowdin(S)
    n = S.shape[0]
    assert np.abs(X - X.T).max() < 1e-13
    assert np.abs(X @ S @ X - np.eye(n)).max() < 1e-10
    assert np.abs(X @ X - np.linalg.inv(S)).max() < 1e-8 * np.abs(np.linalg.inv(S)).max()
    with pytest.raises(LinearDependence):
        lowdin(np.array([[1.0, 1.0], [1.0, 1.0 + 1e-13]]))


# ---------------------------------------------------------------- UHF
@pytest.mark.parametrize("alpha", [0.28, 1.0, 3.7])
def test_uhf_one_electron_single_gaussian(alpha):
    """One electron (H atom, one s Gaussian): the UHF two-electron terms
    J[D^a] - K[D^a] cancel exactly, so E = <T> + <V> =
    3 alpha / 2 - 2 sqrt(2 alpha / pi), and <S^2> = 3/4."""
    m = _pack([1], [[0.2, 0.1, -0.4]], [(0, 0, [alpha], [1.0])], "h", 0, n_electrons=0)
    r = oracle.uhf(m, 1, 0, max_iter=5, e_tol=1e-14)
    assert r.energy == pytest.approx(1.5 * alpha - 2 * math.sqrt(2 * alpha / math.pi), rel=1e-13)
    assert r.s2 == pytest.approx(0.75, abs=1e-14)


def test_uhf_one_electron_is_the_lowest_core_eigenvalue():
    """One electron in an s+p+d basis on three nuclei: no electron-electron
    energy survives, so the UHF energy is the lowest root of the generalised
    eigenproblem H c = e S c plus E_nuc (scipy's LAPACK, a different route)."""
    from scipy.linalg import eigh
    mol = lattice_molecule(3, 3, "spd")
    B = oracle.Basis(mol)
    S, T, V = B.one_electron()
    e0 = eigh(T + V, S, eigvals_only=True)[0]
    r = oracle.uhf(mol, 1, 0, max_iter=10, e_tol=1e-13)
    assert r.energy == pytest.approx(e0 + B.nuclear_repulsion(), abs=1e-10)


@pytest.mark.parametrize("diis", [0, 6])
def test_uhf_closed_shell_equals_rhf(diis):
    """n_alpha = n_beta from the same core guess keeps C^a = C^b, so UHF is
    RHF: same energy (the RHF oracle is pinned above), <S^2> = 0."""
    mol = h_line()
    ro = oracle.rhf(mol, max_iter=80, e_tol=1e-11, diis_size=diis)
    ru = oracle.uhf(mol, 4, 4, max_iter=80, e_tol=1e-11, diis_size=diis)
    assert ru.converged and ru.energy == pytest.approx(ro.energy, abs=1e-9)
    assert abs(ru.s2) < 1e-10
    assert np.abs(ru.Da - ro.D).max() < 1e-6 and np.abs(ru.Db - ro.D).max() < 1e-6


@pytest.mark.parametrize("natom,na,nb", [(5, 3, 2), (6, 4, 2)])
def test_uhf_spin_swap_and_contamination_bound(natom, na, nb):
    """Open shells on an H chain: swapping the alpha and beta counts changes
    neither the energy nor <S^2>, and <S^2> is at least S_z (S_z + 1) (spin
    contamination can only add)."""
    mol = h_line(natom, seed=3)
    r1 = oracle.uhf(mol, na, nb, max_iter=200, e_tol=1e-11, diis_size=6)
    r2 = oracle.uhf(mol, nb, na, max_iter=200, e_tol=1e-11, diis_size=6)
    assert r1.converged and r2.converged
    assert r1.energy == pytest.approx(r2.energy, abs=1e-9)
    assert r1.s2 == pytest.approx(r2.s2, abs=1e-7)
    sz = 0.5 * (na - nb)
    assert r1.s2 >= sz * (sz + 1) - 1e-10


# ---------------------------------------------------------------- MP2
def _spin_orbital_mp2(r, B, n_occ):
    """E(2) = 1/4 sum_{ijab} |<ij||ab>|^2 / (e_i + e_j - e_a - e_b) over spin
    orbitals built from the spatial MOs (the antisymmetrised form), a
    different formula from the oracle's spin-adapted one."""
    G = B.eri_tensor()
    C, eps = r.C, r.eps
    n = C.shape[1]
    mo = np.einsum("pqrs,pi,qj,rk,sl->ijkl", G, C, C, C, C, optimize=True)   # (ij|kl) over spatial MOs
    ns = 2 * n
    spat, spin = np.arange(ns) // 2, np.arange(ns) % 2
    # <pq|rs> = (pr|qs) delta(spin p, spin r) delta(spin q, spin s)
    same = (spin[:, None] == spin[None, :]).astype(float)
    phys = mo[np.ix_(spat, spat, spat, spat)].transpose(0, 2, 1, 3) * same[:, None, :, None] * same[None, :, None, :]
    anti = phys - phys.transpose(0, 1, 3, 2)
    e = eps[spat]
    occ, vir = np.arange(2 * n_occ), np.arange(2 * n_occ, ns)
    A = anti[np.ix_(occ, occ, vir, vir)]
    d = e[occ][:, None, None, None] + e[occ][None, :, None, None] - e[vir][None, None, :, None] - e[vir][None, None, None, :]
    return 0.25 * float(np.sum(A * A / d))


def test_mp2_minimal_basis_h2_closed_form():
    """Minimal-basis H2: one occupied and one virtual orbital, so
    E(2) = K12^2 / (2 (e1 - e2)) with K12 = (12|12) over the MOs."""
    m, _ = _h2()
    B = oracle.Basis(m)
    r = oracle.rhf(m, max_iter=30, e_tol=1e-12)
    G = B.eri_tensor()
    c1, c2 = r.C[:, 0], r.C[:, 1]
    K12 = np.einsum("pqrs,p,q,r,s->", G, c1, c2, c1, c2)
    expect = K12 ** 2 / (2 * (r.eps[0] - r.eps[1]))
    assert oracle.mp2(r, B, 1) == pytest.approx(expect, rel=1e-12)
    assert expect < 0


@pytest.mark.parametrize("mol_fn", [lambda: h_line(6, seed=4), lambda: lattice_molecule(3, 3, "sp")])
def test_mp2_spin_adapted_equals_spin_orbital_form(mol_fn):
    mol = mol_fn()
    B = oracle.Basis(mol)
    r = oracle.rhf(mol, max_iter=100, e_tol=1e-12, diis_size=6)
    n_occ = mol.n_electrons // 2
    assert oracle.mp2(r, B, n_occ) == pytest.approx(_spin_orbital_mp2(r, B, n_occ), rel=1e-10)


def test_mp2_is_size_consistent():
    """Two copies of a molecule far apart: the RHF and MP2 energies are
    twice the single ones up to the dipole-dipole interaction, which falls
    off as R^-3 (checked between 2000 and 10000 bohr).  With identical copies
    the aufbau occupation of the pair is the two single occupations, and the
    canonical MP2 sum is invariant to the mixing of degenerate pair orbitals."""
    a = h_line(4, seed=8)
    ra = oracle.rhf(a, max_iter=100, e_tol=1e-13, diis_size=6)
    e2a = oracle.mp2(ra, oracle.Basis(a), a.n_electrons // 2)
    assert e2a < 0
    d = {}
    for R in (2000.0, 10000.0):
        shells = []
        for k in range(2):
            for s in range(a.nshell):
                p0, n = a.shell_prim[s], a.shell_nprim[s]
                shells.append((int(a.shell_atom[s]) + k * a.natom, int(a.shell_l[s]), a.exps[p0:p0 + n],
                               a.coefs[p0:p0 + n]))
        ab = _pack(np.concatenate([a.Z, a.Z]), np.vstack([a.xyz, a.xyz + np.array([0.0, R, 0.0])]), shells, "ab",
                   0, n_electrons=2 * a.n_electrons)
        r = oracle.rhf(ab, max_iter=100, e_tol=1e-13, diis_size=6)
        d[R] = (r.energy - 2 * ra.energy, oracle.mp2(r, oracle.Basis(ab), a.n_electrons) - 2 * e2a)
    assert abs(d[10000.0][0]) < 1e-10 and abs(d[10000.0][1]) < 1e-11
    for k in range(2):
        assert d[2000.0][k] / d[10000.0][k] == pytest.approx(125.0, rel=0.02)


# ---------------------------------------------------------------- forces
def _h2_one_gaussian_energy():
    """Closed-form RHF energy of H2 with one normalised s Gaussian (exponent
    a) per atom at distance R: the bonding orbital is fixed by symmetry, and
    every integral has a closed form in exp and F_0(t) = sqrt(pi/t) erf(sqrt t)/2,
      E = 2 (h11 + h12) / (1 + S)
          + [(11|11) + (11|22) + 2 (12|12) + 4 (11|12)] / (2 (1 + S)^2) + 1/R."""
    sp = pytest.importorskip("sympy")
    R, a = sp.symbols("R a", positive=True)
    pi = sp.pi

    def F0(t):
        return sp.sqrt(pi / t) * sp.erf(sp.sqrt(t)) / 2
    n2 = (2 * a / pi) ** sp.Rational(3, 2)                 # N^2, N = (2a/pi)^(3/4)
    S = sp.exp(-a * R ** 2 / 2)
    T11, T12 = 3 * a / 2, a / 2 * (3 - a * R ** 2) * S
    v = -(2 * pi / (2 * a)) * n2                           # -(2 pi / p) N^2, p = 2a, unit charge
    V11 = v + v * F0(2 * a * R ** 2)                       # nuclei on A and on B
    V12 = 2 * v * S * F0(2 * a * (R / 2) ** 2)
    g = 2 * pi ** sp.Rational(5, 2) / ((2 * a) ** 2 * sp.sqrt(4 * a)) * n2 ** 2
    A, B = g, g * F0(a * R ** 2)
    C, D = g * sp.exp(-a * R ** 2), g * S * F0(a * R ** 2 / 4)
    E = 2 * (T11 + V11 + T12 + V12) / (1 + S) + (A + B + 2 * C + 4 * D) / (2 * (1 + S) ** 2) + 1 / R
    return sp, R, a, E


@pytest.mark.parametrize("alpha,dist", [(0.8, 1.4), (0.4, 2.2)])
def test_rhf_gradient_matches_the_closed_form_derivative(alpha, dist):
    """dE/dR of the closed form (sympy) against the oracle's gradient, which
    differentiates its own SCF energy; the energies themselves first."""
    sp, R, a, E = _h2_one_gaussian_energy()
    m = _pack([1, 1], [[0, 0, 0], [dist, 0, 0]], [(0, 0, [alpha], [1.0]), (1, 0, [alpha], [1.0])], "h2", 0,
              n_electrons=2)
    e_ref = float(E.subs({R: dist, a: alpha}).evalf(30))
    de_ref = float(sp.diff(E, R).subs({R: dist, a: alpha}).evalf(30))
    assert oracle.rhf(m, max_iter=20, e_tol=1e-13).energy == pytest.approx(e_ref, abs=1e-12)
    g = oracle.rhf_gradient(m)
    assert g[1, 0] == pytest.approx(de_ref, abs=1e-8)
    assert g[0, 0] == pytest.approx(-de_ref, abs=1e-8)
    assert np.abs(g[:, 1:]).max() < 1e-8


def test_rhf_gradient_is_translation_and_rotation_invariant():
    """E does not change under rigid motions, so the gradients sum to zero
    and exert no torque: sum_A g_A = 0, sum_A R_A x g_A = 0."""
    mol = lattice_molecule(4, 5, "sp", charges=(1,), charge_p=(1.0,))   # four H, non-collinear
    g = oracle.rhf_gradient(mol)
    assert np.abs(g).max() > 1e-3
    assert np.abs(g.sum(axis=0)).max() < 1e-7
    assert np.abs(np.cross(mol.xyz, g).sum(axis=0)).max() < 1e-7
