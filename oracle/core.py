"""ctypes binding of the C oracle (``hf_oracle.c``).

TEST INFRASTRUCTURE ONLY (see the package docstring).  The shared object is
compiled with gcc on first use (or by ``build_oracle()``) into
``oracle/_build/``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hf_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build_oracle(force: bool = False) -> str:
    """Compile hf_oracle.c to a shared object (gcc, OpenMP when available)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-fPIC", "-shared", "-std=gnu11", _SRC, "-o", tmp, "-lm"]
    r = subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True, text=True)
    if r.returncode != 0:
        r = subprocess.run(base, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("oracle build failed:\n" + r.stderr)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build_oracle())
        P = C.c_void_p
        i32 = C.c_int
        f64 = C.c_double
        lib.or_boys.restype = f64
        lib.or_boys.argtypes = [i32, f64]
        lib.or_basis_new.restype = P
        lib.or_basis_new.argtypes = [i32, P, P, i32, P, P, P, P, i32, P, P]
        lib.or_basis_free.argtypes = [P]
        lib.or_basis_nbf.restype = i32
        lib.or_basis_nbf.argtypes = [P]
        lib.or_basis_shell_bf.argtypes = [P, P]
        lib.or_one_electron.argtypes = [P, P, P, P]
        lib.or_nuclear_repulsion.restype = f64
        lib.or_nuclear_repulsion.argtypes = [P]
        lib.or_eri.restype = f64
        lib.or_eri.argtypes = [P, i32, i32, i32, i32]
        lib.or_eri_shell_block.argtypes = [P, i32, i32, i32, i32, P]
        lib.or_schwarz.argtypes = [P, P]
        lib.or_eri_tensor.argtypes = [P, P]
        lib.or_jk.restype = C.c_long
        lib.or_jk.argtypes = [P, P, P, P, f64, i32]
        lib.or_jk_rows.argtypes = [P, P, i32, P, P, P, f64, i32]
        lib.or_count_quartets.restype = C.c_long
        lib.or_count_quartets.argtypes = [P, f64]
        lib.or_jk_quartets.argtypes = [P, P, C.c_long, P, P, P]
        lib.or_max_threads.restype = i32
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def boys(m: int, T: float) -> float:
    """F_m(T) = int_0^1 t^(2m) exp(-T t^2) dt (long-double series / erf)."""
    return _load().or_boys(int(m), float(T))


def oracle_threads() -> int:
    """OpenMP threads the oracle would use by default (1 without OpenMP)."""
    return int(_load().or_max_threads())


class Basis:
    """Oracle view of one molecule's basis (normalised contracted Gaussians)."""

    def __init__(self, mol):
        lib = _load()
        self._lib = lib
        self.mol = mol
        self._keep = [np.ascontiguousarray(mol.Z, dtype=np.int32),
                      np.ascontiguousarray(mol.xyz, dtype=np.float64),
                      np.ascontiguousarray(mol.shell_atom, dtype=np.int32),
                      np.ascontiguousarray(mol.shell_l, dtype=np.int32),
                      np.ascontiguousarray(mol.shell_nprim, dtype=np.int32),
                      np.ascontiguousarray(mol.shell_prim, dtype=np.int32),
                      np.ascontiguousarray(mol.exps, dtype=np.float64),
                      np.ascontiguousarray(mol.coefs, dtype=np.float64)]
        Z, xyz, sa, sl, sn, sp, ex, co = self._keep
        h = lib.or_basis_new(int(Z.shape[0]), _ptr(Z), _ptr(xyz), int(sl.shape[0]),
                             _ptr(sa), _ptr(sl), _ptr(sn), _ptr(sp), int(ex.shape[0]),
                             _ptr(ex), _ptr(co))
        if not h:
            raise ValueError("oracle rejected the basis (l > 4, bad indices or nprim < 1)")
        self._h = h
        self.nbf = int(lib.or_basis_nbf(h))
        self.nshell = int(sl.shape[0])
        sbf = np.zeros(self.nshell + 1, dtype=np.int32)
        lib.or_basis_shell_bf(h, _ptr(sbf))
        self.shell_bf = sbf

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.or_basis_free(h)
            self._h = None

    def one_electron(self):
        """(S, T, V) as nbf x nbf float64 arrays (Eqs. 2-4)."""
        n = self.nbf
        S = np.zeros((n, n))
        T = np.zeros((n, n))
        V = np.zeros((n, n))
        self._lib.or_one_electron(self._h, _ptr(S), _ptr(T), _ptr(V))
        return S, T, V

    def nuclear_repulsion(self) -> float:
        return float(self._lib.or_nuclear_repulsion(self._h))

    def eri(self, i, j, k, l) -> float:
        """One contracted integral (ij|kl) over basis functions (Eq. 5)."""
        return float(self._lib.or_eri(self._h, int(i), int(j), int(k), int(l)))

    def eri_shell_block(self, a, b, c, d) -> np.ndarray:
        ls = self.mol.shell_l
        dims = [int((ls[s] + 1) * (ls[s] + 2) // 2) for s in (a, b, c, d)]
        out = np.zeros(dims)
        self._lib.or_eri_shell_block(self._h, int(a), int(b), int(c), int(d), _ptr(out))
        return out

    def eri_tensor(self) -> np.ndarray:
        n = self.nbf
        G = np.zeros((n, n, n, n))
        self._lib.or_eri_tensor(self._h, _ptr(G))
        return G

    def schwarz(self) -> np.ndarray:
        Q = np.zeros((self.nshell, self.nshell))
        self._lib.or_schwarz(self._h, _ptr(Q))
        return Q

    def jk(self, P, tau: float = 0.0, nthreads: int = 1):
        """(J, K, quartets) for density P: J_ij = sum (ij|kl) P_kl,
        K_il = sum (ij|kl) P_jk."""
        P = np.ascontiguousarray(P, dtype=np.float64)
        n = self.nbf
        J = np.zeros((n, n))
        K = np.zeros((n, n))
        cnt = self._lib.or_jk(self._h, _ptr(P), _ptr(J), _ptr(K), float(tau), int(nthreads))
        return J, K, int(cnt)

    def jk_rows(self, P, rows, tau: float = 0.0, nthreads: int = 1):
        P = np.ascontiguousarray(P, dtype=np.float64)
        rows = np.ascontiguousarray(rows, dtype=np.int32)
        n = self.nbf
        Jr = np.zeros((rows.shape[0], n))
        Kr = np.zeros((rows.shape[0], n))
        self._lib.or_jk_rows(self._h, _ptr(P), int(rows.shape[0]), _ptr(rows), _ptr(Jr),
                             _ptr(Kr), float(tau), int(nthreads))
        return Jr, Kr

    def count_quartets(self, tau: float = 0.0) -> int:
        return int(self._lib.or_count_quartets(self._h, float(tau)))

    def jk_quartets(self, P, quads, J=None, K=None):
        """Accumulate the contributions of explicit unique shell quartets."""
        P = np.ascontiguousarray(P, dtype=np.float64)
        q = np.ascontiguousarray(quads, dtype=np.int32).reshape(-1, 4)
        n = self.nbf
        J = np.zeros((n, n)) if J is None else J
        K = np.zeros((n, n)) if K is None else K
        self._lib.or_jk_quartets(self._h, _ptr(P), int(q.shape[0]), _ptr(q), _ptr(J), _ptr(K))
        return J, K
