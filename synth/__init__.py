"""Seeded synthetic molecules and Gaussian basis sets.

This package only draws inputs: nuclear charges, geometries in bohr, shell
layouts, primitive exponents and raw (unnormalised) contraction
coefficients.  It holds none of the Hartree-Fock arithmetic; normalisation,
integrals and SCF live on the two sides that consume these inputs (the CPU
oracle under ``oracle/`` and the CUDA library), each with its own code.
"""
from .molecules import (  # noqa: F401
    water_qz,
    water_cluster_qz,
    small_f_molecule,
    small_g_molecule,
    Molecule,
    h_line,
    lattice_molecule,
    random_shells_molecule,
    batch_molecules,
    serve_stream,
    concat_basis,
    shell_bf_offsets,
    shell_supported_density,
)
