"""GPU path (through the C ABI) against the CPU oracle, element by element.

Tolerances (plain FP64): ERIs and one-electron integrals 1e-12 absolute,
J / K / Fock 1e-10 absolute, SCF energy 1e-8 Eh.
"""
import os

import numpy as np
import pytest

import oracle
from synth import h_line, lattice_molecule, random_shells_molecule

pytestmark = pytest.mark.gpu

ERI_TOL = 1e-12
JK_TOL = 1e-10
E_TOL = 1e-8


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


def _density(n, seed, nocc=None):
    rng = np.random.default_rng(seed)
    C = rng.normal(size=(n, nocc or max(1, n // 3))) / np.sqrt(n)
    return C @ C.T


def _t(x):
    import torch
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda:0")


SPD_CASES = [((0,), 1), ((1, 0), 2), ((1, 1, 0), 3), ((2, 0), 4), ((2, 1, 0), 5), ((2, 2, 1, 0), 6),
             ((2, 1, 2, 0, 1), 7)]


@pytest.mark.parametrize("ls,seed", SPD_CASES)
def test_eri_tensor_all_classes(ctx, hf, ls, seed):
    mol = random_shells_molecule(ls, seed, nprim=(1, 3), exp_range=(0.1, 8.0), box=3.0)
    ob = oracle.Basis(mol)
    G0 = ob.eri_tensor()
    G = hf.Basis(ctx, mol).eri_tensor().cpu().numpy()
    assert np.abs(G - G0).max() <= ERI_TOL


@pytest.mark.parametrize("ls,seed", SPD_CASES[3:])
def test_one_electron(ctx, hf, ls, seed):
    Z = np.arange(1, len(ls) + 1, dtype=np.int32) % 9 + 1
    mol = random_shells_molecule(ls, seed, nprim=(1, 3), exp_range=(0.1, 8.0), box=3.0, Z=Z)
    S0, T0, V0 = oracle.Basis(mol).one_electron()
    S, T, V, en = hf.Basis(ctx, mol).one_electron()
    assert np.abs(S.cpu().numpy() - S0).max() <= ERI_TOL
    assert np.abs(T.cpu().numpy() - T0).max() <= ERI_TOL
    assert np.abs(V.cpu().numpy() - V0).max() <= 1e-11
    assert en == pytest.approx(oracle.Basis(mol).nuclear_repulsion(), abs=1e-12)


@pytest.mark.parametrize("ls,seed", SPD_CASES)
def test_schwarz(ctx, hf, ls, seed):
    mol = random_shells_molecule(ls, seed, nprim=(1, 3), exp_range=(0.1, 8.0), box=3.0)
    Q0 = oracle.Basis(mol).schwarz()
    Q = hf.Basis(ctx, mol).schwarz()
    np.testing.assert_allclose(Q, Q0, rtol=1e-11, atol=1e-14)


@pytest.mark.parametrize("natom,seed,rules", [(3, 1, "sp"), (6, 2, "sp"), (3, 3, "spd"), (9, 4, "s")])
@pytest.mark.parametrize("tau", [0.0, 1e-12])
def test_fock_jk_small(ctx, hf, natom, seed, rules, tau):
    mol = lattice_molecule(natom, seed, rules)
    ob = oracle.Basis(mol)
    D = _density(ob.nbf, seed)
    J0, K0, nq0 = ob.jk(D, tau=tau)
    basis = hf.Basis(ctx, mol)
    J, K = basis.fock_jk(_t(D), opts=hf.jk_opts(schwarz_tau=tau))
    assert np.abs(J.cpu().numpy() - J0).max() <= JK_TOL
    assert np.abs(K.cpu().numpy() - K0).max() <= JK_TOL
    nq, _ = basis.count_quartets(hf.jk_opts(schwarz_tau=tau))
    assert abs(nq - nq0) <= max(2, nq0 // 10000)   # Schwarz ties at the threshold may differ


def test_fock_jk_host_pointers_match_device(ctx, hf):
    mol = lattice_molecule(5, 9, "sp")
    basis = hf.Basis(ctx, mol)
    D = _density(basis.nbf, 1)
    J, K = basis.fock_jk(_t(D))
    Jh, Kh = basis.fock_jk(D)   # numpy -> HF_JK_HOST path
    assert np.abs(Jh - J.cpu().numpy()).max() <= 1e-13
    assert np.abs(Kh - K.cpu().numpy()).max() <= 1e-13


def test_fock_jk_ragged_many_tiles(ctx, hf):
    # enough pairs per class for many 32-ket work items with ragged tails
    mol = lattice_molecule(10, 21, "sp")
    ob = oracle.Basis(mol)
    D = _density(ob.nbf, 5)
    J0, K0, _ = ob.jk(D, tau=1e-12, nthreads=oracle.oracle_threads())
    J, K = hf.Basis(ctx, mol).fock_jk(_t(D))
    assert np.abs(J.cpu().numpy() - J0).max() <= JK_TOL
    assert np.abs(K.cpu().numpy() - K0).max() <= JK_TOL


def test_scf_h_line_stored_and_direct(ctx, hf):
    mol = h_line()
    ro = oracle.rhf(mol, max_iter=30, e_tol=1e-8, diis_size=0)
    basis = hf.Basis(ctx, mol)
    for stored in (False, True):
        r = basis.scf(max_iter=30, e_tol=1e-8, diis_size=0, schwarz_tau=0.0, stored_eri=stored)
        assert r.converged == ro.converged
        assert abs(r.energy - ro.energy) <= E_TOL
        assert np.abs(r.tensors["F1"].cpu().numpy() - ro.F1).max() <= JK_TOL
    G = basis.eri_tensor()
    D = _t(ro.D)
    J, K = basis.jk_stored(G, D)
    J0, K0, _ = oracle.Basis(mol).jk(ro.D)
    assert np.abs(J.cpu().numpy() - J0).max() <= JK_TOL
    assert np.abs(K.cpu().numpy() - K0).max() <= JK_TOL


@pytest.mark.parametrize("natom,seed,rules", [(4, 31, "sp"), (6, 32, "sp"), (3, 33, "spd")])
def test_scf_diis_small(ctx, hf, natom, seed, rules):
    mol = lattice_molecule(natom, seed, rules)
    ro = oracle.rhf(mol, max_iter=128, e_tol=1e-8, diis_size=8, tau=1e-12, nthreads=oracle.oracle_threads())
    r = hf.Basis(ctx, mol).scf(max_iter=128, e_tol=1e-8, diis_size=8, schwarz_tau=1e-12)
    assert r.converged == ro.converged
    assert abs(r.energy - ro.energy) <= E_TOL
    if ro.homo_lumo_gap > 1e-8:
        assert np.abs(r.tensors["D"].cpu().numpy() - ro.D).max() <= 1e-6
    assert np.abs(r.tensors["F1"].cpu().numpy() - ro.F1).max() <= JK_TOL


def test_c2_full_size_sampled_rows(ctx, hf):
    """40-atom s+p lattice (the benchmark workload): J/K rows against the
    oracle's row-wise definition, in the launch configuration the benchmark
    times (Schwarz tau 1e-12, FP64).  The density is supported on a random
    subset of 16 shells so that the oracle's rows stay cheap; the GPU still
    evaluates every surviving quartet."""
    mol = lattice_molecule(40, 1, "sp")
    ob = oracle.Basis(mol)
    rng = np.random.default_rng(78)
    shells = np.sort(rng.choice(mol.nshell, size=16, replace=False))
    idx = np.concatenate([np.arange(ob.shell_bf[s], ob.shell_bf[s + 1]) for s in shells])
    C = np.zeros((ob.nbf, 8))
    C[idx] = rng.normal(size=(idx.size, 8)) / np.sqrt(idx.size)
    D = C @ C.T
    basis = hf.Basis(ctx, mol)
    J, K = basis.fock_jk(_t(D))
    J = J.cpu().numpy()
    K = K.cpu().numpy()
    rows = np.array([0, 57, 101, int(idx[3]), ob.nbf - 1])
    Jr, Kr = ob.jk_rows(D, rows, tau=1e-12, nthreads=oracle.oracle_threads())
    assert np.abs(J[rows] - Jr).max() <= JK_TOL
    assert np.abs(K[rows] - Kr).max() <= JK_TOL
    assert np.abs(J - J.T).max() == 0.0 and np.abs(K - K.T).max() == 0.0
    assert np.abs(Kr).max() > 1e-3 and np.abs(Jr).max() > 1e-3


@pytest.mark.slow
@pytest.mark.skipif(not os.environ.get("HF_FULL_C3"),
                    reason="two full 150-atom s+p+d J/K builds take about 20 GPU-minutes; set HF_FULL_C3=1")
def test_c3_full_size_rows_against_stored_oracle(ctx, hf):
    """150-atom s+p+d lattice (nbf 1366, K 1..6) at full size, Schwarz tau
    1e-12: FP64 and df64 J/K rows against oracle rows stored in
    tests/golden/c3_rows.npz.  tests/golden/make_c3_rows.py wrote them by
    calling only the oracle (about 5 CPU-minutes on 8 x86 cores, far longer
    on a host whose long double is software quad precision), so they are
    stored rather than recomputed.  The density is supported on six shells,
    two of them d; the GPU evaluates every surviving quartet of the molecule
    (1.45e10 after Schwarz screening: 757 s per FP64 build on one GB300)."""
    from synth import shell_supported_density
    gold = np.load(os.path.join(os.path.dirname(__file__), "golden", "c3_rows.npz"))
    mol = lattice_molecule(150, 2, "spd")
    D, shells, rows = shell_supported_density(mol, seed=11)
    assert gold["rows"].tolist() == rows.tolist() and gold["shells"].tolist() == list(shells)
    basis = hf.Basis(ctx, mol)
    assert basis.nbf == 1366
    for o in (hf.jk_opts(schwarz_tau=1e-12), hf.jk_opts(schwarz_tau=1e-12, df64=True)):
        J, K = basis.fock_jk(_t(D), opts=o)
        J = J.cpu().numpy()
        K = K.cpu().numpy()
        assert np.abs(J[rows] - gold["J"]).max() <= JK_TOL
        assert np.abs(K[rows] - gold["K"]).max() <= JK_TOL
        assert np.abs(J - J.T).max() == 0.0 and np.abs(K - K.T).max() == 0.0
    assert np.abs(gold["K"]).max() > 1e-2 and np.abs(gold["J"]).max() > 1e-2


@pytest.mark.parametrize("natom,seed,rules", [(9, 41, "sp"), (3, 3, "spd")])
def test_fp32_split_error_is_bounded(ctx, hf, natom, seed, rules):
    mol = lattice_molecule(natom, seed, rules)
    ob = oracle.Basis(mol)
    D = _density(ob.nbf, 9, nocc=mol.n_electrons // 2)
    J0, K0, _ = ob.jk(D, tau=1e-12, nthreads=oracle.oracle_threads())
    basis = hf.Basis(ctx, mol)
    nq, nf = basis.count_quartets(hf.jk_opts(fp32_bound=1e-5))
    assert 0 < nf < nq or rules == "spd"
    for boys32 in (False, True):
        J, K = basis.fock_jk(_t(D), opts=hf.jk_opts(fp32_bound=1e-5, fp32_boys=boys32))
        dj = np.abs(J.cpu().numpy() - J0).max()
        dk = np.abs(K.cpu().numpy() - K0).max()
        assert dj <= 1e-7 and dk <= 1e-7, (dj, dk)


@pytest.mark.parametrize("natom,seed,rules", [(6, 2, "sp"), (3, 3, "spd"), (9, 4, "s")])
def test_df64_tier_matches_oracle(ctx, hf, natom, seed, rules):
    """Double-float (FP32-pair) arithmetic for the quartets above the FP32
    bound, in every class (the s+p+d cases reach the warp-cooperative
    kernels of L >= 5): J/K within the FP64 tolerance of the oracle."""
    mol = lattice_molecule(natom, seed, rules)
    ob = oracle.Basis(mol)
    D = _density(ob.nbf, seed)
    J0, K0, _ = ob.jk(D, tau=1e-12, nthreads=oracle.oracle_threads())
    basis = hf.Basis(ctx, mol)
    for fb in (0.0, 1e-5):
        J, K = basis.fock_jk(_t(D), opts=hf.jk_opts(fp32_bound=fb, df64=True))
        tol = JK_TOL if fb == 0.0 else 1e-7
        assert np.abs(J.cpu().numpy() - J0).max() <= tol
        assert np.abs(K.cpu().numpy() - K0).max() <= tol


def test_df64_cooperative_classes_match_fp64(ctx, hf):
    """12-atom s+p+d molecule: the df64 form of every class, the
    warp-cooperative L >= 5 ones included, against the FP64 path (itself
    oracle-pinned above) within the FP64 J/K tolerance."""
    mol = lattice_molecule(12, 3, "spd")
    basis = hf.Basis(ctx, mol)
    D = _t(_density(basis.nbf, 12, nocc=mol.n_electrons // 2))
    J64, K64 = basis.fock_jk(D)
    Jd, Kd = basis.fock_jk(D, opts=hf.jk_opts(df64=True))
    assert float((Jd - J64).abs().max()) <= JK_TOL
    assert float((Kd - K64).abs().max()) <= JK_TOL
    heavy = [st for st in basis.class_stats(hf.jk_opts()) if st.la + st.lb + st.lc + st.ld >= 5]
    assert sum(st.quartets_fp64 for st in heavy) > 0


def test_df64_full_size_and_scf(ctx, hf):
    """40-atom workload: df64 J/K against the FP64 path; SCF energies with
    df64 against FP64 and the oracle-pinned small case."""
    mol = lattice_molecule(40, 1, "sp")
    basis = hf.Basis(ctx, mol)
    D = _t(_density(basis.nbf, 5, nocc=mol.n_electrons // 2))
    J64, K64 = basis.fock_jk(D)
    Jd, Kd = basis.fock_jk(D, opts=hf.jk_opts(df64=True))
    assert float((Jd - J64).abs().max()) <= JK_TOL
    assert float((Kd - K64).abs().max()) <= JK_TOL
    small = lattice_molecule(6, 32, "sp")
    ro = oracle.rhf(small, max_iter=128, e_tol=1e-8, diis_size=8, tau=1e-12, nthreads=oracle.oracle_threads())
    r = hf.Basis(ctx, small).scf(max_iter=128, e_tol=1e-8, diis_size=8, df64=True)
    assert abs(r.energy - ro.energy) <= E_TOL


def test_errors(ctx, hf):
    mol = lattice_molecule(3, 1, "sp")
    odd = hf.Basis(ctx, mol, n_electrons=3)      # a basis takes any count; closed-shell RHF does not
    with pytest.raises(hf.HFError) as e:
        odd.scf()
    assert e.value.code == -8
    bad = mol.copy()
    bad.shell_l = bad.shell_l.copy()
    bad.shell_l[0] = 5   # above HF_LMAX (g)
    with pytest.raises(hf.HFError) as e:
        hf.Basis(ctx, bad)
    assert e.value.code == -2
    bad = mol.copy()
    bad.exps = bad.exps.copy()
    bad.exps[0] = -1.0
    with pytest.raises(hf.HFError) as e:
        hf.Basis(ctx, bad)
    assert e.value.code == -1
    # linear dependence: the same shell twice on one atom
    from synth.molecules import _pack
    dup = _pack([1, 1], [[0, 0, 0], [1.4, 0, 0]], [(0, 0, [1.0], [1.0]), (0, 0, [1.0], [1.0]), (1, 0, [1.0], [1.0])],
                "dup", 0, n_electrons=2)
    r = hf.Basis(ctx, dup)
    with pytest.raises(hf.HFError) as e:
        r.scf()
    assert e.value.code == -4


def test_not_converged_reports_partial(ctx, hf):
    mol = lattice_molecule(4, 31, "sp")
    r = hf.Basis(ctx, mol).scf(max_iter=1, diis_size=0)
    assert r.rc == -5 and not r.converged and r.iterations == 1 and np.isfinite(r.energy)


def test_injected_allocation_failure(ctx, hf):
    mol = lattice_molecule(4, 5, "sp")
    ctx.inject_alloc_failure(3)
    with pytest.raises(hf.HFError) as e:
        hf.Basis(ctx, mol)
    assert e.value.code == -3
    ctx.inject_alloc_failure(0)
    hf.Basis(ctx, mol)   # context still usable


def test_single_function_and_zero_electrons(ctx, hf):
    from synth.molecules import _pack
    m = _pack([2], [[0.0, 0.0, 0.0]], [(0, 0, [0.7671], [1.0])], "he", 0, n_electrons=2)
    r = hf.Basis(ctx, m).scf(max_iter=5, e_tol=1e-12)
    a = 0.7671
    ref = 3 * a - 8 * np.sqrt(2 * a / np.pi) + 2 * np.sqrt(a / np.pi)
    assert abs(r.energy - ref) <= 1e-12
    m0 = lattice_molecule(3, 1, "sp")
    b0 = hf.Basis(ctx, m0, n_electrons=0)
    D = _density(b0.nbf, 1) * 0.0
    J, K = b0.fock_jk(_t(D))
    assert float(J.abs().max()) == 0.0 and float(K.abs().max()) == 0.0


def test_deterministic_jk_is_bitwise_reproducible(ctx, hf):
    """HF_JK_DETERMINISTIC: the fixed-point accumulation gives the same bits
    on every call (FP64 atomics do not), matches the default build and the
    oracle within the J/K tolerance, for RHF and unrestricted J/K, and every
    precision tier."""
    import torch
    mol = lattice_molecule(6, 21, "spd")
    basis = hf.Basis(ctx, mol)
    ob = oracle.Basis(mol)
    n = basis.nbf
    rng = np.random.default_rng(5)
    Cm = rng.normal(size=(n, 4)) / np.sqrt(n)
    Dn = Cm @ Cm.T
    Jr, Kr, _ = ob.jk(Dn, tau=1e-12, nthreads=oracle.oracle_threads())
    D = torch.tensor(Dn, device="cuda:0")
    for tier in ({}, {"df64": True}, {"fp32_bound": 1e-5, "df64": True}):
        Jd, Kd = basis.fock_jk(D, opts=hf.jk_opts(deterministic=True, **tier))
        for _ in range(3):
            J2, K2 = basis.fock_jk(D, opts=hf.jk_opts(deterministic=True, **tier))
            assert torch.equal(J2, Jd) and torch.equal(K2, Kd), tier
        tol = JK_TOL if "fp32_bound" not in tier else 1e-7
        assert np.abs(Jd.cpu().numpy() - Jr).max() <= tol and np.abs(Kd.cpu().numpy() - Kr).max() <= tol, tier
    Db = D * 0.5
    a = basis.fock_jk_uhf(D, Db, opts=hf.jk_opts(deterministic=True))
    b = basis.fock_jk_uhf(D, Db, opts=hf.jk_opts(deterministic=True))
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    assert float((a[0] - torch.tensor(1.5 * Jr, device="cuda:0")).abs().max()) <= JK_TOL
    import ctypes
    from paper_1303_4916_gb300 import _abi
    o = hf.hf_scf_opts_default()                         # the SCF does not take the flag
    o.jk = hf.jk_opts(deterministic=True)
    r = _abi.hf_scf_result()
    assert hf.load().hf_scf_solve(basis.handle, ctypes.byref(o), ctypes.byref(r)) == _abi.HF_ERR_INVALID


def test_scf_iteration_log(ctx, hf, tmp_path):
    """hf_ctx_set_log: one JSON line per SCF iteration (RHF and UHF) with the
    energy sequence the solve reports."""
    import json
    path = tmp_path / "scf.jsonl"
    c = hf.Context(0)
    c.set_log(str(path))
    mol = lattice_molecule(3, 51, "sp")
    b = hf.Basis(c, mol)
    r = b.scf(max_iter=64, e_tol=1e-9, diis_size=8)
    u = b.uhf(mol.n_electrons // 2 + 1, mol.n_electrons // 2 - 1, max_iter=64, e_tol=1e-9)
    c.set_log(None)
    lines = [json.loads(x) for x in path.read_text().splitlines()]
    rhf = [x for x in lines if x["solver"] == "rhf"]
    uhf = [x for x in lines if x["solver"] == "uhf"]
    assert len(rhf) == r.iterations and len(uhf) == u.iterations
    assert [x["iter"] for x in rhf] == list(range(1, r.iterations + 1))
    assert rhf[0]["delta_e"] is None and rhf[-1]["converged"] == int(r.converged)
    assert abs(rhf[-1]["energy"] - r.energy) <= 1e-12 and abs(uhf[-1]["energy"] - u.energy) <= 1e-12
    assert all(x["nbf"] == b.nbf and x["t"] >= 0.0 for x in lines)


def test_context_outlived_by_its_bases(hf):
    """A context destroyed while bases and a server made on it are alive
    stays usable by them; the last of them completes the teardown (the order
    a garbage collector may pick at interpreter exit)."""
    import torch
    lib = hf.load()
    c = hf.Context(0)
    mol = lattice_molecule(3, 51, "sp")
    b1 = hf.Basis(c, mol)
    b2 = hf.Basis(c, mol)
    srv = hf.Server(c, max_active=2)
    c.close()                                             # destroy pending: three users alive
    D = torch.eye(b1.nbf, dtype=torch.float64, device="cuda:0") * 0.1
    J, K = b1.fock_jk(D)
    torch.cuda.synchronize()
    assert torch.isfinite(J).all() and torch.isfinite(K).all()
    b1.close()
    srv.close()
    e = b2.scf(max_iter=64).energy                       # still works
    assert np.isfinite(e)
    b2.close()                                            # the last user: teardown happens here
    from paper_1303_4916_gb300 import _abi
    assert lib.hf_strerror(_abi.HF_OK) is not None


def test_scf_restart_from_density(ctx, hf):
    """Checkpoint / resume: an SCF started from a converged density (D0)
    lands on the same energy within two iterations."""
    mol = lattice_molecule(6, 32, "sp")
    b = hf.Basis(ctx, mol)
    r = b.scf(max_iter=128, e_tol=1e-10, diis_size=8)
    assert r.converged
    r2 = b.scf(max_iter=128, e_tol=1e-10, diis_size=8, D0=r.tensors["D"])
    assert r2.converged and r2.iterations <= 3
    assert abs(r2.energy - r.energy) <= 1e-9


def _max_prim_atom(nprim, seed):
    """One atom carrying an s and a p shell of nprim primitives and a d shell
    of three (exponents log-uniform in [0.05, 50], coefficients U[0.2, 1])."""
    from synth.molecules import _pack
    rng = np.random.default_rng(seed)
    shells = []
    for l, k in ((0, nprim), (1, nprim), (2, 3)):
        e = np.exp(rng.uniform(np.log(0.05), np.log(50.0), k))
        shells.append((0, l, list(e), list(rng.uniform(0.2, 1.0, k))))
    return _pack([8], [[0.1, -0.2, 0.3]], shells, "maxprim", seed, n_electrons=8)


def test_single_centre_and_maximum_primitives(ctx, hf):
    """Edge cases of the integral path against the oracle: all four centres of
    every quartet coincide (one atom with s, p and d shells: A - B = C - D =
    P - Q = 0, Boys argument T = 0) and the s and p shells have the maximum of
    HF_MAX_NPRIM primitives (16^4 primitive quartets in (pp|pp), the longest
    primitive loops the kernels and their split items see), for the ERI
    tensor, J/K in the FP64 and df64 tiers and the Schwarz factors; one
    primitive more is refused."""
    from paper_1303_4916_gb300 import _abi
    mol = _max_prim_atom(_abi.HF_MAX_NPRIM, 5)
    ob = oracle.Basis(mol)
    b = hf.Basis(ctx, mol)
    G = b.eri_tensor().cpu().numpy()
    assert np.abs(G - ob.eri_tensor()).max() <= ERI_TOL
    assert np.allclose(b.schwarz(), ob.schwarz(), rtol=1e-11, atol=1e-14)
    D = _density(ob.nbf, 9)
    J0, K0, _ = ob.jk(D, tau=0.0, nthreads=oracle.oracle_threads())
    for tier in ({}, {"df64": True}):
        J, K = b.fock_jk(_t(D), opts=hf.jk_opts(schwarz_tau=0.0, **tier))
        assert np.abs(J.cpu().numpy() - J0).max() <= JK_TOL, tier
        assert np.abs(K.cpu().numpy() - K0).max() <= JK_TOL, tier
    with pytest.raises(hf.HFError) as e:
        hf.Basis(ctx, _max_prim_atom(_abi.HF_MAX_NPRIM + 1, 5))
    assert e.value.code == _abi.HF_ERR_INVALID
