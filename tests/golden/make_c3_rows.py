#!/usr/bin/env python3
"""Write c3_rows.npz: oracle J/K rows of the 150-atom s+p+d lattice molecule
(seed 2) for a seeded density supported on six shells, Schwarz tau 1e-12.

Calls only the CPU oracle (oracle/) and the seeded input generators
(synth/); bench.py's c3check workload and the GPU test draw the same input.
Usage: python tests/golden/make_c3_rows.py
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from synth import lattice_molecule, shell_supported_density  # noqa: E402


def main():
    mol = lattice_molecule(150, 2, "spd")
    ob = oracle.Basis(mol)
    D, shells, rows = shell_supported_density(mol, seed=11)
    t0 = time.time()
    Jr, Kr = ob.jk_rows(D, rows, tau=1e-12, nthreads=oracle.oracle_threads())
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c3_rows.npz")
    np.savez_compressed(out, rows=rows, shells=np.array(shells), J=Jr, K=Kr)
    print(f"wrote {out} ({time.time() - t0:.0f} s, {oracle.oracle_threads()} threads)")


if __name__ == "__main__":
    main()
