"""Rys-quadrature route (Eq. 5 by Rys quadrature, the paper's own route) on
the GPU against the CPU oracle (McMurchie-Davidson, independent of both
GPU routes): every class with an f or g shell, the one-electron integrals
of f/g shells, Schwarz factors, J/K with and without screening, the
HF_JK_RYS switch that routes the s/p/d classes through the same kernel,
and RHF energies, including H2O in a quadruple-zeta-shaped basis (the
shape of the paper's HF timing benchmark) against a stored oracle energy.

Tolerances as for the Obara-Saika route: ERIs and one-electron integrals
1e-12 absolute, J/K 1e-10, SCF energy 1e-8 Eh.
"""
import json
import os

import numpy as np
import pytest

import oracle
from synth import lattice_molecule, random_shells_molecule, small_f_molecule, water_qz

pytestmark = pytest.mark.gpu

ERI_TOL = 1e-12
JK_TOL = 1e-10
E_TOL = 1e-8
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def hf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1303_4916_gb300 as hf
    return hf


@pytest.fixture(scope="module")
def ctx(hf):
    return hf.Context(0)


def _t(x):
    import torch
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda:0")


def _density(n, seed, nocc=None):
    rng = np.random.default_rng(seed)
    C = rng.normal(size=(n, nocc or max(1, n // 3))) / np.sqrt(n)
    return C @ C.T


# shells per case, one atom each: every f/g pair class appears as bra and
# as ket, (gg|gg) included; primitives per shell kept small where the
# oracle's tensor would be slow
FG_CASES = [((3,), 1, (1, 3)), ((3, 0), 2, (1, 3)), ((3, 1, 0), 3, (1, 3)), ((4, 0), 4, (1, 3)),
            ((3, 2, 1), 5, (1, 3)), ((4, 3), 6, (1, 1)), ((4, 2, 0, 1), 7, (1, 2)), ((4, 4), 8, (1, 1)),
            ((3, 3, 2), 9, (1, 2))]


def test_eri_tensor_fg_far_apart(ctx, hf):
    """Centres ~10 bohr apart with tight exponents: T = pq/(p+q) |PQ|^2 well
    above 60, where the rule takes its Gauss-Hermite limit."""
    mol = random_shells_molecule((3, 2, 4), 10, nprim=(1, 2), exp_range=(2.0, 8.0), box=14.0)
    G0 = oracle.Basis(mol).eri_tensor()
    G = hf.Basis(ctx, mol).eri_tensor().cpu().numpy()
    assert np.abs(G - G0).max() <= ERI_TOL


@pytest.mark.parametrize("ls,seed,nprim", FG_CASES)
def test_eri_tensor_fg_classes(ctx, hf, ls, seed, nprim):
    mol = random_shells_molecule(ls, seed, nprim=nprim, exp_range=(0.2, 6.0), box=2.5)
    G0 = oracle.Basis(mol).eri_tensor()
    G = hf.Basis(ctx, mol).eri_tensor().cpu().numpy()
    assert np.abs(G - G0).max() <= ERI_TOL


@pytest.mark.parametrize("ls,seed,nprim", FG_CASES)
def test_schwarz_fg(ctx, hf, ls, seed, nprim):
    mol = random_shells_molecule(ls, seed, nprim=nprim, exp_range=(0.2, 6.0), box=2.5)
    Q0 = oracle.Basis(mol).schwarz()
    Q = hf.Basis(ctx, mol).schwarz()
    np.testing.assert_allclose(Q, Q0, rtol=1e-11, atol=1e-14)


@pytest.mark.parametrize("ls,seed,nprim", FG_CASES[2:])
def test_one_electron_fg(ctx, hf, ls, seed, nprim):
    Z = np.arange(1, len(ls) + 1, dtype=np.int32) % 9 + 2
    mol = random_shells_molecule(ls, seed, nprim=nprim, exp_range=(0.2, 6.0), box=2.5, Z=Z)
    S0, T0, V0 = oracle.Basis(mol).one_electron()
    S, T, V, _ = hf.Basis(ctx, mol).one_electron()
    assert np.abs(S.cpu().numpy() - S0).max() <= ERI_TOL
    assert np.abs(T.cpu().numpy() - T0).max() <= ERI_TOL
    assert np.abs(V.cpu().numpy() - V0).max() <= 1e-11


@pytest.mark.parametrize("tau", [0.0, 1e-12])
def test_fock_jk_fg_molecule(ctx, hf, tau):
    ls = (4, 3, 2, 1, 0, 3, 1, 0)
    mol = random_shells_molecule(ls, 21, nprim=(1, 2), exp_range=(0.15, 5.0), box=4.0)
    ob = oracle.Basis(mol)
    D = _density(ob.nbf, 4)
    J0, K0, nq0 = ob.jk(D, tau=tau, nthreads=oracle.oracle_threads())
    basis = hf.Basis(ctx, mol)
    J, K = basis.fock_jk(_t(D), opts=hf.jk_opts(schwarz_tau=tau))
    assert np.abs(J.cpu().numpy() - J0).max() <= JK_TOL
    assert np.abs(K.cpu().numpy() - K0).max() <= JK_TOL
    nq, _ = basis.count_quartets(hf.jk_opts(schwarz_tau=tau))
    assert abs(nq - nq0) <= max(2, nq0 // 10000)
    # the f/g classes run the FP64 Rys kernel in every precision mode
    for o in (hf.jk_opts(schwarz_tau=tau, df64=True), hf.jk_opts(schwarz_tau=tau, rys=True)):
        J2, K2 = basis.fock_jk(_t(D), opts=o)
        assert np.abs(J2.cpu().numpy() - J0).max() <= JK_TOL
        assert np.abs(K2.cpu().numpy() - K0).max() <= JK_TOL


@pytest.mark.parametrize("natom,seed,rules", [(3, 1, "sp"), (3, 3, "spd"), (9, 4, "s")])
def test_rys_route_for_every_class_matches_oracle(ctx, hf, natom, seed, rules):
    """HF_JK_RYS: the s/p/d classes through the Rys kernel instead of the
    Obara-Saika / Head-Gordon-Pople ones; same J/K as the oracle."""
    mol = lattice_molecule(natom, seed, rules)
    ob = oracle.Basis(mol)
    D = _density(ob.nbf, seed)
    J0, K0, _ = ob.jk(D, tau=1e-12, nthreads=oracle.oracle_threads())
    basis = hf.Basis(ctx, mol)
    J, K = basis.fock_jk(_t(D), opts=hf.jk_opts(rys=True))
    assert np.abs(J.cpu().numpy() - J0).max() <= JK_TOL
    assert np.abs(K.cpu().numpy() - K0).max() <= JK_TOL
    # the FP32-tagged list goes through the same FP64 Rys kernel
    J2, K2 = basis.fock_jk(_t(D), opts=hf.jk_opts(rys=True, fp32_bound=1e-5))
    assert np.abs(J2.cpu().numpy() - J0).max() <= JK_TOL
    assert np.abs(K2.cpu().numpy() - K0).max() <= JK_TOL


def test_deterministic_fg_is_bitwise_reproducible(ctx, hf):
    ls = (4, 3, 1, 0, 2)
    mol = random_shells_molecule(ls, 31, nprim=(1, 2), exp_range=(0.2, 5.0), box=3.0)
    basis = hf.Basis(ctx, mol)
    D = _t(_density(basis.nbf, 7))
    J1, K1 = basis.fock_jk(D, opts=hf.jk_opts(deterministic=True))
    J2, K2 = basis.fock_jk(D, opts=hf.jk_opts(deterministic=True))
    assert (J1 == J2).all() and (K1 == K2).all()
    J0, K0 = basis.fock_jk(D)
    assert (J1 - J0).abs().max().item() <= 1e-12
    assert (K1 - K0).abs().max().item() <= 1e-12


def test_scf_with_f_shells_matches_oracle(ctx, hf):
    Z = np.array([8, 1, 6, 1], dtype=np.int32)
    mol = random_shells_molecule((0, 0, 1, 3), 41, nprim=(2, 3), exp_range=(0.2, 4.0), box=3.0, Z=Z)
    # one more contracted s shell per atom keeps the basis complete enough
    from synth.molecules import _pack
    shells = []
    for s in range(mol.nshell):
        o, k = mol.shell_prim[s], mol.shell_nprim[s]
        shells.append((int(mol.shell_atom[s]), int(mol.shell_l[s]), mol.exps[o:o + k], mol.coefs[o:o + k]))
    for a in range(mol.natom):
        shells.append((a, 0, np.array([0.3, 1.5, 7.0]), np.array([0.5, 0.4, 0.2])))
    mol = _pack(mol.Z, mol.xyz, shells, "fshells", 41)
    ro = oracle.rhf(mol, max_iter=128, e_tol=1e-9, diis_size=8, tau=1e-12, nthreads=oracle.oracle_threads())
    r = hf.Basis(ctx, mol).scf(max_iter=128, e_tol=1e-9, diis_size=8, schwarz_tau=1e-12)
    assert r.converged and ro.converged
    assert abs(r.energy - ro.energy) <= E_TOL


def test_water_qz_energy_and_rows(ctx, hf):
    """H2O, synthetic quadruple-zeta-shaped basis (nbf 140, up to g): RHF
    energy against the stored oracle energy, and J/K rows of a seeded
    density against the oracle."""
    ref = json.load(open(os.path.join(GOLDEN, "water_qz.json")))
    mol = water_qz(0)
    basis = hf.Basis(ctx, mol)
    r = basis.scf(max_iter=100, e_tol=1e-10, diis_size=8, schwarz_tau=0.0)
    assert r.converged
    assert abs(r.energy - ref["energy"]) <= E_TOL
    D = _density(basis.nbf, 9, nocc=5)
    rows = [0, 27, 69, 70, 139]
    Jr, Kr = oracle.Basis(mol).jk_rows(D, rows, tau=0.0, nthreads=oracle.oracle_threads())
    J, K = basis.fock_jk(_t(D), opts=hf.jk_opts(schwarz_tau=0.0))
    assert np.abs(J.cpu().numpy()[rows] - Jr).max() <= JK_TOL
    assert np.abs(K.cpu().numpy()[rows] - Kr).max() <= JK_TOL


def test_batch_with_fg_molecule_matches_single(ctx, hf):
    mols = [random_shells_molecule((3, 1, 0, 0), 51, nprim=(1, 2), exp_range=(0.3, 4.0), box=3.0,
                                   Z=np.array([2, 2, 1, 1], dtype=np.int32)),
            lattice_molecule(3, 1, "sp")]
    bases = [hf.Basis(ctx, m) for m in mols]
    single = [b.scf(max_iter=128, e_tol=1e-9, diis_size=8) for b in bases]
    batch, status = hf.scf_solve_batch(bases, max_iter=128, e_tol=1e-9, diis_size=8)
    assert status == [0, 0]
    for s, b in zip(single, batch):
        assert abs(s.energy - b.energy) <= 1e-9


def test_uhf_jk_fg_matches_oracle(ctx, hf):
    """One integral evaluation feeding J[Da + Db], K[Da] and K[Db] through the
    Rys kernels (warp and thread forms) against the oracle."""
    mol = random_shells_molecule((4, 3, 1, 0, 2), 71, nprim=(1, 2), exp_range=(0.2, 5.0), box=3.5)
    ob = oracle.Basis(mol)
    Da, Db = _density(ob.nbf, 1), _density(ob.nbf, 2)
    J0, _, _ = ob.jk(Da + Db, tau=0.0, nthreads=oracle.oracle_threads())
    _, Ka0, _ = ob.jk(Da, tau=0.0, nthreads=oracle.oracle_threads())
    _, Kb0, _ = ob.jk(Db, tau=0.0, nthreads=oracle.oracle_threads())
    J, Ka, Kb = hf.Basis(ctx, mol).fock_jk_uhf(_t(Da), _t(Db), opts=hf.jk_opts(schwarz_tau=0.0))
    assert np.abs(J.cpu().numpy() - J0).max() <= JK_TOL
    assert np.abs(Ka.cpu().numpy() - Ka0).max() <= JK_TOL
    assert np.abs(Kb.cpu().numpy() - Kb0).max() <= JK_TOL


def test_uhf_with_f_shells_matches_oracle(ctx, hf):
    mol = small_f_molecule(0)   # 8 electrons: a triplet, 5 alpha and 3 beta
    ro = oracle.uhf(mol, 5, 3, max_iter=200, e_tol=1e-10, diis_size=8, tau=0.0)
    r = hf.Basis(ctx, mol).uhf(5, 3, max_iter=200, e_tol=1e-10, diis_size=8, schwarz_tau=0.0)
    assert r.converged and ro.converged
    assert abs(r.energy - ro.energy) <= E_TOL
