"""GB300 (sm_103a) library for the closed-shell Hartree-Fock two-electron hot
path: contracted Cartesian Gaussian ERIs (Eq. 5) contracted into J and K
(the J/K equation of Sec. "Technical details"), the RHF and UHF iterations
around it, and batched / continuous-batching serving forms.

The compute lives in ``libhf.so`` (CUDA, C ABI in ``include/hf.h``); this
package is its ctypes binding.  The first call loads the library and raises
if it has not been built: there is no CPU fallback.
"""
from . import _abi  # noqa: F401
from .api import (  # noqa: F401
    hf_basis_create,
    hf_count_quartets,
    hf_ctx_create,
    hf_eri_tensor,
    hf_fock_jk,
    hf_fock_jk_uhf,
    hf_fock_jk_noalloc,
    hf_jk_stored,
    hf_mp2_energy,
    hf_one_electron,
    hf_rhf_gradient,
    hf_rys_rule,
    hf_scf_solve,
    hf_scf_solve_batch,
    hf_schwarz,
    hf_serve_cancel,
    hf_serve_create,
    hf_serve_drain,
    hf_serve_poll,
    hf_serve_submit,
    hf_uhf_solve,
    Basis,
    Context,
    HFError,
    SCFResult,
    Server,
    UHFResult,
    hf_jk_opts_default,
    hf_scf_opts_default,
    jk_opts,
    scf_solve_batch,
)


def load():
    """Load libhf.so (raises ImportError when it is missing)."""
    return _abi.load()
