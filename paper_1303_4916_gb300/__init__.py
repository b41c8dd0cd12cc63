"""GB300 (sm_103a) library for the closed-shell Hartree-Fock two-electron hot
path: contracted Cartesian Gaussian ERIs (Eq. 5) contracted into J and K
(the J/K equation of Sec. "Technical details"), the RHF iteration around
it, and batched / continuous-batching serving forms.

The compute lives in ``libhf.so`` (CUDA, C ABI in ``include/hf.h``); this
package is its ctypes binding.  Importing the binding loads the library and
raises if it has not been built: there is no CPU fallback.
"""
from . import _abi  # noqa: F401
from .api import (  # noqa: F401
    Basis,
    Context,
    HFError,
    SCFResult,
    Server,
    hf_jk_opts_default,
    hf_scf_opts_default,
    jk_opts,
    scf_solve_batch,
)


def load():
    """Load libhf.so (raises ImportError when it is missing)."""
    return _abi.load()
