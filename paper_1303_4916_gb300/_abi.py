"""ctypes declarations of the C ABI in include/hf.h (argument marshalling only).

The shared library ``libhf.so`` must have been built (``build.build()``);
loading fails loudly otherwise -- there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# HF_LIB selects another build of the same ABI, e.g. the bounds-checked
# libhf_bcheck.so (paper_1303_4916_gb300.build.build_bounds_checked())
LIB_PATH = os.environ.get("HF_LIB") or os.path.join(HERE, "libhf.so")

HF_OK = 0
HF_PENDING = 1
HF_ERR_INVALID = -1
HF_ERR_UNSUPPORTED_L = -2
HF_ERR_OOM = -3
HF_ERR_LINDEP = -4
HF_ERR_NOT_CONVERGED = -5
HF_ERR_TIMEOUT = -6
HF_ERR_CUDA = -7
HF_ERR_ODD_ELECTRONS = -8
HF_ERR_NOT_FOUND = -9
HF_ERR_QUEUE_FULL = -10
HF_ERR_CANCELLED = -11
HF_ERR_TOO_LARGE = -12
HF_LMAX = 4
HF_MAX_NPRIM = 16
HF_STORED_NBF_MAX = 400

HF_JK_HOST = 1
HF_JK_DETERMINISTIC = 2
HF_JK_FP32_BOYS = 4
HF_JK_DF64 = 8
HF_JK_RYS = 16
HF_SCF_STORED_ERI = 1


class hf_atom(C.Structure):
    _fields_ = [("Z", C.c_int), ("xyz", C.c_double * 3)]


class hf_shell(C.Structure):
    _fields_ = [("atom", C.c_int), ("l", C.c_int), ("nprim", C.c_int), ("prim_off", C.c_int)]


class hf_jk_opts(C.Structure):
    _fields_ = [("schwarz_tau", C.c_double), ("fp32_bound", C.c_double), ("flags", C.c_uint)]


class hf_scf_opts(C.Structure):
    _fields_ = [("max_iter", C.c_int), ("e_tol", C.c_double), ("diis_size", C.c_int),
                ("D0", C.c_void_p), ("jk", hf_jk_opts), ("flags", C.c_uint)]


class hf_scf_result(C.Structure):
    _fields_ = [("energy", C.c_double), ("e_elec", C.c_double), ("e_nuc", C.c_double),
                ("delta_e", C.c_double), ("diis_error", C.c_double), ("homo_lumo_gap", C.c_double),
                ("iterations", C.c_int), ("converged", C.c_int), ("fock_builds", C.c_longlong),
                ("quartets", C.c_longlong), ("seconds", C.c_double),
                ("D", C.c_void_p), ("C", C.c_void_p), ("eps", C.c_void_p), ("F", C.c_void_p),
                ("F1", C.c_void_p)]


class hf_uhf_result(C.Structure):
    _fields_ = [("energy", C.c_double), ("e_elec", C.c_double), ("e_nuc", C.c_double),
                ("delta_e", C.c_double), ("diis_error", C.c_double), ("s2", C.c_double),
                ("iterations", C.c_int), ("converged", C.c_int), ("fock_builds", C.c_longlong),
                ("quartets", C.c_longlong), ("seconds", C.c_double),
                ("Da", C.c_void_p), ("Db", C.c_void_p), ("eps_a", C.c_void_p), ("eps_b", C.c_void_p)]


class hf_class_stats(C.Structure):
    _fields_ = [("la", C.c_int), ("lb", C.c_int), ("lc", C.c_int), ("ld", C.c_int),
                ("vrr_flops", C.c_int), ("hrr_flops", C.c_int), ("prim_flops", C.c_int),
                ("digest_flops", C.c_int),
                ("quartets_fp64", C.c_longlong), ("prim_quartets_fp64", C.c_longlong),
                ("quartets_fp32", C.c_longlong), ("prim_quartets_fp32", C.c_longlong)]


HF_NCLASS = 120


class hf_serve_opts(C.Structure):
    _fields_ = [("max_active", C.c_int), ("queue_capacity", C.c_int), ("hbm_budget", C.c_size_t),
                ("scf", hf_scf_opts)]


class hf_request(C.Structure):
    _fields_ = [("atoms", C.POINTER(hf_atom)), ("natom", C.c_int), ("shells", C.POINTER(hf_shell)),
                ("nshell", C.c_int), ("exps", C.POINTER(C.c_double)), ("coefs", C.POINTER(C.c_double)),
                ("nprim", C.c_int), ("n_electrons", C.c_int)]


class hf_serve_result(C.Structure):
    _fields_ = [("status", C.c_int), ("energy", C.c_double), ("iterations", C.c_int),
                ("converged", C.c_int), ("nbf", C.c_int), ("t_submit", C.c_double),
                ("t_admit", C.c_double), ("t_done", C.c_double), ("fock_builds", C.c_longlong),
                ("quartets", C.c_longlong)]


P = C.c_void_p
I = C.c_int
D = C.c_double

# name: (restype, argtypes) -- one line per declaration of include/hf.h
SIGNATURES = {
    "hf_jk_opts_default": (None, [C.POINTER(hf_jk_opts)]),
    "hf_scf_opts_default": (None, [C.POINTER(hf_scf_opts)]),
    "hf_strerror": (C.c_char_p, [I]),
    "hf_last_error": (C.c_char_p, []),
    "hf_ctx_create": (I, [C.POINTER(P), I, C.c_size_t, P]),
    "hf_ctx_destroy": (None, [P]),
    "hf_ctx_stream": (P, [P]),
    "hf_ctx_num_sms": (I, [P]),
    "hf_ctx_inject_alloc_failure": (None, [P, I]),
    "hf_ctx_set_log": (I, [P, C.c_char_p]),
    "hf_bounds_checked": (I, []),
    "hf_basis_create": (I, [P, C.POINTER(hf_atom), I, C.POINTER(hf_shell), I, P, P, I, C.POINTER(P)]),
    "hf_basis_destroy": (None, [P]),
    "hf_basis_nbf": (I, [P]),
    "hf_basis_nshell": (I, [P]),
    "hf_basis_device_bytes": (C.c_size_t, [P]),
    "hf_schwarz": (I, [P, P]),
    "hf_count_quartets": (I, [P, C.POINTER(hf_jk_opts), C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]),
    "hf_fock_jk": (I, [P, P, P, P, C.POINTER(hf_jk_opts)]),
    "hf_class_stats_get": (I, [P, C.POINTER(hf_jk_opts), C.POINTER(hf_class_stats)]),
    "hf_fock_jk_profiled": (I, [P, P, P, P, C.POINTER(hf_jk_opts), C.POINTER(C.c_double)]),
    "hf_fock_jk_noalloc": (I, [P, P, P, P, C.POINTER(hf_jk_opts)]),
    "hf_one_electron": (I, [P, P, P, P, C.POINTER(D)]),
    "hf_eri_tensor": (I, [P, P]),
    "hf_jk_stored": (I, [P, P, P, P, P]),
    "hf_scf_solve": (I, [P, C.POINTER(hf_scf_opts), C.POINTER(hf_scf_result)]),
    "hf_fock_jk_uhf": (I, [P, P, P, P, P, P, C.POINTER(hf_jk_opts)]),
    "hf_uhf_solve": (I, [P, I, I, C.POINTER(hf_scf_opts), C.POINTER(hf_uhf_result)]),
    "hf_mp2_energy": (I, [P, P, P, I, C.POINTER(D)]),
    "hf_rys_rule": (I, [I, D, C.POINTER(D), C.POINTER(D)]),
    "hf_rhf_gradient": (I, [P, P, P, I, P, C.POINTER(D)]),
    "hf_scf_solve_batch": (I, [C.POINTER(P), I, C.POINTER(hf_scf_opts), C.POINTER(hf_scf_result),
                               C.POINTER(I)]),
    "hf_serve_opts_default": (None, [C.POINTER(hf_serve_opts)]),
    "hf_serve_create": (I, [P, C.POINTER(hf_serve_opts), C.POINTER(P)]),
    "hf_serve_submit": (I, [P, C.POINTER(hf_request), C.POINTER(C.c_uint64)]),
    "hf_serve_poll": (I, [P, C.c_uint64, C.POINTER(hf_serve_result)]),
    "hf_serve_cancel": (I, [P, C.c_uint64]),
    "hf_serve_now": (D, [P]),
    "hf_serve_drain": (I, [P, D]),
    "hf_serve_destroy": (None, [P]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libhf.so and declare every entry point; raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libhf.so not built at {path}: run paper_1303_4916_gb300.build.build()")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
