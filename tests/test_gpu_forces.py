"""Analytic RHF nuclear gradient (the paper's Hartree-Fock forces) on the GPU
against the oracle's gradient, which differentiates the oracle's converged
energy numerically (tests/golden/make_gradients.py; pinned in
test_oracle_pins.py against a closed-form derivative and the translation and
rotation invariances).

Tolerance 1e-6 Eh/bohr: the analytic gradient at an SCF converged to
|dE| <= 1e-12 against a Richardson-extrapolated central difference (error
O(h^4) with h = 2e-3 bohr, energies converged to 1e-13).
"""
import json
import os

import numpy as np
import pytest

from synth import h_line, lattice_molecule, small_f_molecule, small_g_molecule

pytestmark = pytest.mark.gpu

G_TOL = 1e-6
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "gradients.json")
MOLS = {
    "h_line2": lambda: h_line(2, seed=0),
    "lattice3_sp": lambda: lattice_molecule(3, 1, "sp"),
    "lattice3_spd": lambda: lattice_molecule(3, 3, "spd"),
    "small_f": lambda: small_f_molecule(0),
    "small_g": lambda: small_g_molecule(0),
}


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


@pytest.fixture(scope="module")
def golden():
    return json.load(open(GOLDEN))["cases"]


@pytest.mark.parametrize("name", list(MOLS))
def test_gradient_matches_oracle(ctx, hf, golden, name):
    mol = MOLS[name]()
    ref = golden[name]
    basis = hf.Basis(ctx, mol)
    r = basis.scf(max_iter=200, e_tol=1e-12, diis_size=8, schwarz_tau=0.0)
    assert r.converged
    assert abs(r.energy - ref["energy"]) <= 1e-8
    g = basis.gradient(r, schwarz_tau=0.0)
    g0 = np.asarray(ref["gradient"])
    assert np.abs(g - g0).max() <= G_TOL, (g, g0)
    # translational invariance: the forces on all atoms add up to zero
    assert np.abs(g.sum(axis=0)).max() <= 1e-9


def test_gradient_with_screening_and_after_jk(ctx, hf, golden):
    """Schwarz screening at 1e-12 moves the gradient by far less than the
    tolerance; J/K builds before and after (work lists of either shape) stay
    correct."""
    mol = MOLS["lattice3_spd"]()
    basis = hf.Basis(ctx, mol)
    r = basis.scf(max_iter=200, e_tol=1e-12, diis_size=8)
    D = r.tensors["D"]
    J0, K0 = basis.fock_jk(D)
    g = basis.gradient(r, schwarz_tau=1e-12)
    assert np.abs(g - np.asarray(golden["lattice3_spd"]["gradient"])).max() <= G_TOL
    J1, K1 = basis.fock_jk(D)
    assert (J1 - J0).abs().max().item() <= 1e-12 and (K1 - K0).abs().max().item() <= 1e-12


def test_gradient_rejects_bad_arguments(ctx, hf):
    import ctypes
    mol = MOLS["h_line2"]()
    basis = hf.Basis(ctx, mol)
    r = basis.scf()
    lib = hf.api._lib()
    g = (ctypes.c_double * 6)()
    Cp = ctypes.c_void_p(r.tensors["C"].data_ptr())
    ep = ctypes.c_void_p(r.tensors["eps"].data_ptr())
    assert lib.hf_rhf_gradient(basis.handle, Cp, ep, 0, None, g) == -1
    assert lib.hf_rhf_gradient(basis.handle, Cp, ep, 3, None, g) == -1
    assert lib.hf_rhf_gradient(basis.handle, None, ep, 1, None, g) == -1
