"""MP2 correlation energy on the GPU (the paper's MP2, Szabo-Ostlund's
closed-shell formula over canonical orbitals) against the oracle's mp2:
with the oracle's own orbitals as input (the transform and the sum alone),
and end to end from the GPU's RHF."""
import json
import os

import numpy as np
import pytest

import oracle
from synth import h_line, lattice_molecule

pytestmark = pytest.mark.gpu


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


CASES = [("H8 chain", lambda: h_line()), ("s+p", lambda: lattice_molecule(3, 51, "sp")),
         ("s+p+d", lambda: lattice_molecule(2, 101, "spd"))]


@pytest.mark.parametrize("name,make", CASES)
def test_mp2_matches_oracle(ctx, hf, name, make):
    import torch
    mol = make()
    ob = oracle.Basis(mol)
    ro = oracle.rhf(mol, max_iter=128, e_tol=1e-11, diis_size=8, tau=0.0, nthreads=oracle.oracle_threads(),
                    basis=ob)
    assert ro.converged
    no = mol.n_electrons // 2
    e_ref = oracle.mp2(ro, ob, no)
    basis = hf.Basis(ctx, mol)
    # the oracle's orbitals through the GPU transform: only the arithmetic differs
    C = torch.tensor(np.ascontiguousarray(ro.C), device="cuda:0")
    eps = torch.tensor(np.ascontiguousarray(ro.eps), device="cuda:0")
    e_gpu = basis.mp2_energy(C, eps, no)
    assert abs(e_gpu - e_ref) <= 1e-11 * max(1.0, abs(e_ref)), (name, e_gpu, e_ref)
    # end to end: the GPU's RHF orbitals (converged to the same tolerance)
    r = basis.scf(max_iter=128, e_tol=1e-11, diis_size=8, schwarz_tau=0.0)
    assert r.converged
    e_e2e = basis.mp2_energy(r.tensors["C"], r.tensors["eps"], no)
    assert abs(e_e2e - e_ref) <= 1e-8, (name, e_e2e, e_ref)
    assert e_ref < 0.0


def test_mp2_rejects_bad_arguments(ctx, hf):
    import torch
    from paper_1303_4916_gb300 import _abi
    basis = hf.Basis(ctx, h_line())
    n = basis.nbf
    C = torch.eye(n, dtype=torch.float64, device="cuda:0")
    eps = torch.arange(n, dtype=torch.float64, device="cuda:0")
    for no in (0, n):
        with pytest.raises(hf.HFError) as e:
            basis.mp2_energy(C, eps, no)
        assert e.value.code == _abi.HF_ERR_INVALID


def test_mp2_and_stored_eri_beyond_128_functions(ctx, hf):
    """nbf 140 (28 nuclei with one f, d, p or s shell each, so the Rys
    classes too): the AO tensor (3.1 GB) held in HBM for the MP2 transform
    and for the stored-ERI SCF, against the oracle's energies
    (tests/golden/make_mp2_large.py)."""
    from synth import random_shells_molecule
    ref = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "mp2_large.json")))
    mol = random_shells_molecule([3, 2, 1, 0] * 7, 4, nprim=(1, 1), exp_range=(0.3, 3.0), box=10.0)
    basis = hf.Basis(ctx, mol)
    assert basis.nbf == ref["nbf"] > 128
    r = basis.scf(max_iter=128, e_tol=1e-11, diis_size=8, schwarz_tau=0.0)
    assert r.converged and abs(r.energy - ref["energy"]) <= 1e-8
    e2 = basis.mp2_energy(r.tensors["C"], r.tensors["eps"], mol.n_electrons // 2)
    assert abs(e2 - ref["e_mp2"]) <= 1e-8, (e2, ref["e_mp2"])
    rs = basis.scf(max_iter=128, e_tol=1e-11, diis_size=8, schwarz_tau=0.0, stored_eri=True, outputs=False)
    assert rs.converged and abs(rs.energy - ref["energy"]) <= 1e-8
