#!/usr/bin/env python3
"""Write mp2_large.json: the oracle's converged RHF energy and MP2
correlation energy of 28 hydrogen nuclei carrying one single-primitive
shell each, f, d, p, s repeated (synth.random_shells_molecule, seed 4, box
10 bohr; nbf 140, above the sizes the stored-tensor paths were first built
for), DIIS 8, e_tol 1e-11, no screening.

Calls only the CPU oracle (oracle/) and the seeded input generators
(synth/).  Usage: python tests/golden/make_mp2_large.py
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from synth import random_shells_molecule  # noqa: E402


def molecule():
    return random_shells_molecule([3, 2, 1, 0] * 7, 4, nprim=(1, 1), exp_range=(0.3, 3.0), box=10.0)


def main():
    mol = molecule()
    t0 = time.time()
    ob = oracle.Basis(mol)
    r = oracle.rhf(mol, max_iter=128, e_tol=1e-11, diis_size=8, tau=0.0, nthreads=oracle.oracle_threads(), basis=ob)
    no = mol.n_electrons // 2
    e2 = oracle.mp2(r, ob, no)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "mp2_large.json")
    with open(out, "w") as fh:
        json.dump({"molecule": "synth.random_shells_molecule([3, 2, 1, 0] * 7, 4, nprim=(1, 1), "
                               "exp_range=(0.3, 3.0), box=10.0)", "nbf": mol.nbf, "n_occ": no,
                   "energy": r.energy, "iterations": r.iterations, "converged": bool(r.converged),
                   "homo_lumo_gap": r.homo_lumo_gap, "e_mp2": e2, "e_tol": 1e-11, "diis_size": 8, "tau": 0.0},
                  fh, indent=1)
    print(f"wrote {out}: E = {r.energy:.12f}, E(2) = {e2:.12f} ({time.time() - t0:.0f} s)")


if __name__ == "__main__":
    main()
