#!/usr/bin/env python3
"""Write water_qz.json: the oracle's converged RHF energy of H2O in the
synthetic quadruple-zeta-shaped basis (synth.water_qz, seed 0: s, p, d, f
and g shells, nbf 140) -- the shape of the paper's HF timing benchmark
(H2O, Fig. 4) -- with Pulay DIIS (8 vectors), e_tol 1e-10 and Schwarz tau 0.

Calls only the CPU oracle (oracle/) and the seeded input generators
(synth/).  Usage: python tests/golden/make_water_qz.py
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from synth import water_qz  # noqa: E402


def main():
    mol = water_qz(0)
    t0 = time.time()
    r = oracle.rhf(mol, max_iter=100, e_tol=1e-10, diis_size=8, tau=0.0, nthreads=oracle.oracle_threads())
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "water_qz.json")
    with open(out, "w") as fh:
        json.dump({"molecule": "synth.water_qz(0)", "nbf": mol.nbf, "energy": r.energy,
                   "iterations": r.iterations, "converged": bool(r.converged),
                   "homo_lumo_gap": r.homo_lumo_gap, "e_tol": 1e-10, "diis_size": 8, "tau": 0.0}, fh, indent=1)
    print(f"wrote {out}: E = {r.energy:.12f} ({r.iterations} it, {time.time() - t0:.0f} s)")


if __name__ == "__main__":
    main()
