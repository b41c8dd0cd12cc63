#!/usr/bin/env python3
"""Write gradients.json: the oracle's RHF nuclear gradients (central
differences of its converged energy at steps 2e-3 and 1e-3 bohr, Richardson
extrapolated; oracle.rhf_gradient) for the molecules the GPU force tests
use: a 2-atom H chain (s), a 3-atom s+p lattice molecule, a 3-atom s+p+d
lattice molecule, an O-H pair with an f shell and one with a g shell.

Calls only the CPU oracle (oracle/) and the seeded input generators
(synth/).  Usage: python tests/golden/make_gradients.py
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from synth import h_line, lattice_molecule, small_f_molecule, small_g_molecule  # noqa: E402

CASES = {
    "h_line2": lambda: h_line(2, seed=0),
    "lattice3_sp": lambda: lattice_molecule(3, 1, "sp"),
    "lattice3_spd": lambda: lattice_molecule(3, 3, "spd"),
    "small_f": lambda: small_f_molecule(0),
    "small_g": lambda: small_g_molecule(0),
}


def main():
    out = {}
    for name, make in CASES.items():
        t0 = time.time()
        mol = make()
        g = oracle.rhf_gradient(mol)
        r = oracle.rhf(mol, max_iter=200, e_tol=1e-13, diis_size=8)
        out[name] = {"gradient": g.tolist(), "energy": r.energy, "natom": mol.natom, "nbf": mol.nbf}
        print(f"{name}: {time.time() - t0:.0f} s", flush=True)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "gradients.json")
    with open(path, "w") as fh:
        json.dump({"method": "oracle.rhf_gradient (h = 2e-3, Richardson), e_tol 1e-13, DIIS 8", "cases": out}, fh,
                  indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
