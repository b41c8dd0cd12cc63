"""CPU oracle for closed-shell Hartree-Fock (test infrastructure).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the library under
``paper_1303_4916_gb300/`` never does, and this package never imports it.

``Basis`` wraps the plain C implementation in ``hf_oracle.c`` (integrals,
Boys function, J/K); ``rhf`` and ``uhf`` in ``scf.py`` run the textbook RHF
and unrestricted (Pople-Nesbet) iterations on top of it with numpy, and
``mp2`` the second-order Moller-Plesset energy of an RHF solution, and
``rhf_gradient`` the nuclear gradient of the RHF energy.
"""
from .core import Basis, boys, build_oracle, oracle_threads  # noqa: F401
from .scf import mp2, rhf, rhf_gradient, uhf, RHFResult, UHFResult, LinearDependence  # noqa: F401
