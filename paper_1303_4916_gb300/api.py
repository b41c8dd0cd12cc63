"""Thin Python binding of libhf (include/hf.h).

Every call below marshals arguments and calls the C ABI; all arithmetic of
the hot path runs in the CUDA library.  PyTorch provides device memory and
streams: matrices are passed as raw data pointers of contiguous float64
CUDA tensors on the context's device.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass
from typing import Optional

import numpy as np

from . import _abi
from ._abi import (hf_atom, hf_shell, hf_jk_opts, hf_scf_opts, hf_scf_result, hf_serve_opts,
                   hf_request, hf_serve_result)


class HFError(RuntimeError):
    def __init__(self, code: int, where: str):
        lib = _abi.load()
        msg = lib.hf_last_error().decode(errors="replace")
        name = lib.hf_strerror(code).decode()
        super().__init__(f"{where}: {name} ({code}): {msg}")
        self.code = code


def _check(rc: int, where: str, ok=(_abi.HF_OK,)):
    if rc not in ok:
        raise HFError(rc, where)
    return rc


def _lib():
    return _abi.load()


def _ptr(t) -> int:
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch tensor")
    if t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError("expected a contiguous float64 tensor")
    return t.data_ptr()


def hf_jk_opts_default() -> hf_jk_opts:
    o = hf_jk_opts()
    _lib().hf_jk_opts_default(C.byref(o))
    return o


def hf_scf_opts_default() -> hf_scf_opts:
    o = hf_scf_opts()
    _lib().hf_scf_opts_default(C.byref(o))
    return o


def jk_opts(schwarz_tau: Optional[float] = None, fp32_bound: Optional[float] = None, host: bool = False,
            fp32_boys: bool = False, df64: bool = False, deterministic: bool = False,
            rys: bool = False) -> hf_jk_opts:
    o = hf_jk_opts_default()
    if rys:
        o.flags |= _abi.HF_JK_RYS
    if deterministic:
        o.flags |= _abi.HF_JK_DETERMINISTIC
    if schwarz_tau is not None:
        o.schwarz_tau = schwarz_tau
    if fp32_bound is not None:
        o.fp32_bound = fp32_bound
    if host:
        o.flags |= _abi.HF_JK_HOST
    if fp32_boys:
        o.flags |= _abi.HF_JK_FP32_BOYS
    if df64:
        o.flags |= _abi.HF_JK_DF64
    return o


class Context:
    """hf_ctx on one CUDA device; by default ordered on torch's current stream."""

    def __init__(self, device: int = 0, hbm_budget: int = 0, stream=None, use_torch_stream: bool = True):
        import torch
        lib = _lib()
        self._h = C.c_void_p()
        if stream is None and use_torch_stream:
            torch.cuda.set_device(device)
            stream = torch.cuda.current_stream(device).cuda_stream
        _check(lib.hf_ctx_create(C.byref(self._h), device, hbm_budget, stream), "hf_ctx_create")
        self.device = device

    @property
    def handle(self):
        return self._h

    @property
    def num_sms(self) -> int:
        return _lib().hf_ctx_num_sms(self._h)

    def inject_alloc_failure(self, n: int):
        _lib().hf_ctx_inject_alloc_failure(self._h, n)

    def set_log(self, path: Optional[str]):
        """JSON-lines log of every SCF iteration ("-" = stderr, None = off)."""
        _check(_lib().hf_ctx_set_log(self._h, None if path is None else path.encode()), "hf_ctx_set_log")

    def close(self):
        if self._h:
            _lib().hf_ctx_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _marshal(mol):
    """(atoms, shells, exps, coefs) ctypes arrays from a molecule-like object
    with Z, xyz, shell_atom, shell_l, shell_nprim, shell_prim, exps, coefs."""
    na = int(len(mol.Z))
    atoms = (hf_atom * na)()
    for i in range(na):
        atoms[i].Z = int(mol.Z[i])
        for x in range(3):
            atoms[i].xyz[x] = float(mol.xyz[i][x])
    ns = int(len(mol.shell_l))
    shells = (hf_shell * ns)()
    for s in range(ns):
        shells[s].atom = int(mol.shell_atom[s])
        shells[s].l = int(mol.shell_l[s])
        shells[s].nprim = int(mol.shell_nprim[s])
        shells[s].prim_off = int(mol.shell_prim[s])
    exps = np.ascontiguousarray(mol.exps, dtype=np.float64)
    coefs = np.ascontiguousarray(mol.coefs, dtype=np.float64)
    return atoms, shells, exps, coefs


class Basis:
    """hf_basis of one molecule (device-resident shell-pair data)."""

    def __init__(self, ctx: Context, mol, n_electrons: Optional[int] = None):
        lib = _lib()
        atoms, shells, exps, coefs = _marshal(mol)
        ne = int(mol.n_electrons if n_electrons is None else n_electrons)
        self._h = C.c_void_p()
        _check(lib.hf_basis_create(ctx.handle, atoms, len(atoms), shells, len(shells),
                                   exps.ctypes.data_as(C.c_void_p), coefs.ctypes.data_as(C.c_void_p), ne,
                                   C.byref(self._h)), "hf_basis_create")
        self.ctx = ctx
        self.nbf = lib.hf_basis_nbf(self._h)
        self.nshell = lib.hf_basis_nshell(self._h)
        self.n_electrons = ne
        self.natom = len(atoms)

    @property
    def handle(self):
        return self._h

    def device_bytes(self) -> int:
        return int(_lib().hf_basis_device_bytes(self._h))

    def close(self):
        if self._h:
            _lib().hf_basis_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def schwarz(self) -> np.ndarray:
        Q = np.zeros((self.nshell, self.nshell))
        _check(_lib().hf_schwarz(self._h, Q.ctypes.data_as(C.c_void_p)), "hf_schwarz")
        return Q

    def count_quartets(self, opts: Optional[hf_jk_opts] = None):
        n, f = C.c_longlong(), C.c_longlong()
        _check(_lib().hf_count_quartets(self._h, C.byref(opts) if opts else None, C.byref(n), C.byref(f)),
               "hf_count_quartets")
        return int(n.value), int(f.value)

    def fock_jk(self, D, J=None, K=None, opts: Optional[hf_jk_opts] = None):
        """J, K for the density D (CUDA tensors, or numpy arrays with a host-flagged opts)."""
        import torch
        if isinstance(D, np.ndarray):
            o = opts if opts is not None else jk_opts()
            o.flags |= _abi.HF_JK_HOST
            Dh = np.ascontiguousarray(D, dtype=np.float64)
            Jh = np.empty_like(Dh) if J is None else J
            Kh = np.empty_like(Dh) if K is None else K
            _check(_lib().hf_fock_jk(self._h, Dh.ctypes.data_as(C.c_void_p), Jh.ctypes.data_as(C.c_void_p),
                                     Kh.ctypes.data_as(C.c_void_p), C.byref(o)), "hf_fock_jk")
            return Jh, Kh
        if J is None:
            J = torch.empty_like(D)
        if K is None:
            K = torch.empty_like(D)
        _check(_lib().hf_fock_jk(self._h, _ptr(D), _ptr(J), _ptr(K), C.byref(opts) if opts else None),
               "hf_fock_jk")
        return J, K

    def fock_jk_host(self, D_ptr: int, J_ptr: int, K_ptr: int, opts: hf_jk_opts):
        """Raw-pointer form (host buffers with HF_JK_HOST, e.g. pinned tensors)."""
        return _check(_lib().hf_fock_jk(self._h, D_ptr, J_ptr, K_ptr, C.byref(opts)), "hf_fock_jk")

    def class_stats(self, opts: Optional[hf_jk_opts] = None):
        arr = (_abi.hf_class_stats * _abi.HF_NCLASS)()
        _check(_lib().hf_class_stats_get(self._h, C.byref(opts) if opts else None, arr), "hf_class_stats_get")
        return list(arr)

    def fock_jk_profiled(self, D, J, K, opts: Optional[hf_jk_opts] = None):
        """hf_fock_jk with per-class kernel durations (ms): array [HF_NCLASS, 2] (fp64, fp32)."""
        ms = (C.c_double * (2 * _abi.HF_NCLASS))()
        _check(_lib().hf_fock_jk_profiled(self._h, _ptr(D), _ptr(J), _ptr(K), C.byref(opts) if opts else None, ms),
               "hf_fock_jk_profiled")
        return np.array(list(ms)).reshape(_abi.HF_NCLASS, 2)

    def one_electron(self):
        import torch
        n = self.nbf
        dev = torch.device("cuda", self.ctx.device)
        S, T, V = (torch.empty((n, n), dtype=torch.float64, device=dev) for _ in range(3))
        en = C.c_double()
        _check(_lib().hf_one_electron(self._h, _ptr(S), _ptr(T), _ptr(V), C.byref(en)), "hf_one_electron")
        return S, T, V, float(en.value)

    def eri_tensor(self):
        import torch
        n = self.nbf
        G = torch.empty((n, n, n, n), dtype=torch.float64, device=torch.device("cuda", self.ctx.device))
        _check(_lib().hf_eri_tensor(self._h, _ptr(G)), "hf_eri_tensor")
        return G

    def jk_stored(self, G, D):
        import torch
        J = torch.empty_like(D)
        K = torch.empty_like(D)
        _check(_lib().hf_jk_stored(self._h, _ptr(G), _ptr(D), _ptr(J), _ptr(K)), "hf_jk_stored")
        return J, K

    def scf(self, max_iter: int = 128, e_tol: float = 1e-8, diis_size: int = 8, schwarz_tau: float = 1e-12,
            fp32_bound: float = 0.0, stored_eri: bool = False, D0=None, outputs: bool = True,
            allow_unconverged: bool = True, fp32_boys: bool = False, df64: bool = False):
        import torch
        o = hf_scf_opts_default()
        o.max_iter = max_iter
        o.e_tol = e_tol
        o.diis_size = diis_size
        o.jk = jk_opts(schwarz_tau, fp32_bound, fp32_boys=fp32_boys, df64=df64)
        if stored_eri:
            o.flags |= _abi.HF_SCF_STORED_ERI
        if D0 is not None:
            o.D0 = _ptr(D0)
        r = hf_scf_result()
        out = {}
        if outputs:
            n = self.nbf
            dev = torch.device("cuda", self.ctx.device)
            for k in ("D", "C", "F", "F1"):
                out[k] = torch.empty((n, n), dtype=torch.float64, device=dev)
                setattr(r, k, out[k].data_ptr())
            out["eps"] = torch.empty((n,), dtype=torch.float64, device=dev)
            r.eps = out["eps"].data_ptr()
        ok = (_abi.HF_OK, _abi.HF_ERR_NOT_CONVERGED) if allow_unconverged else (_abi.HF_OK,)
        rc = _check(_lib().hf_scf_solve(self._h, C.byref(o), C.byref(r)), "hf_scf_solve", ok)
        return SCFResult(rc=rc, energy=r.energy, e_elec=r.e_elec, e_nuc=r.e_nuc, delta_e=r.delta_e,
                         diis_error=r.diis_error, homo_lumo_gap=r.homo_lumo_gap, iterations=r.iterations,
                         converged=bool(r.converged), fock_builds=r.fock_builds, quartets=r.quartets,
                         seconds=r.seconds, tensors=out)

    def mp2_energy(self, Cmo, eps, n_occ: int) -> float:
        """E(2) from MO coefficients Cmo[mu][p] and ascending orbital energies eps (CUDA tensors)."""
        e2 = C.c_double()
        _check(_lib().hf_mp2_energy(self._h, _ptr(Cmo), _ptr(eps), int(n_occ), C.byref(e2)), "hf_mp2_energy")
        return float(e2.value)

    def gradient(self, scf_result=None, schwarz_tau: float = 1e-12, e_tol: float = 1e-11):
        """Analytic RHF gradient dE/dR (numpy natom x 3, Eh/bohr) at the
        converged density of scf_result (a tight SCF is run when none is
        given); the forces are its negative."""
        r = scf_result if scf_result is not None else self.scf(e_tol=e_tol, schwarz_tau=schwarz_tau)
        g = np.zeros((self.natom, 3))
        o = jk_opts(schwarz_tau)
        _check(_lib().hf_rhf_gradient(self._h, _ptr(r.tensors["C"]), _ptr(r.tensors["eps"]),
                                      int(self.n_electrons // 2), C.byref(o),
                                      g.ctypes.data_as(C.POINTER(C.c_double))), "hf_rhf_gradient")
        return g

    def fock_jk_uhf(self, Da, Db, opts: Optional[hf_jk_opts] = None):
        """J[Da + Db], K[Da], K[Db] (CUDA tensors) from one integral evaluation."""
        import torch
        J, Ka, Kb = torch.empty_like(Da), torch.empty_like(Da), torch.empty_like(Da)
        _check(_lib().hf_fock_jk_uhf(self._h, _ptr(Da), _ptr(Db), _ptr(J), _ptr(Ka), _ptr(Kb),
                                     C.byref(opts) if opts else None), "hf_fock_jk_uhf")
        return J, Ka, Kb

    def uhf(self, n_alpha: int, n_beta: int, max_iter: int = 128, e_tol: float = 1e-8, diis_size: int = 8,
            schwarz_tau: float = 1e-12, fp32_bound: float = 0.0, df64: bool = False, outputs: bool = True,
            allow_unconverged: bool = True):
        import torch
        o = hf_scf_opts_default()
        o.max_iter = max_iter
        o.e_tol = e_tol
        o.diis_size = diis_size
        o.jk = jk_opts(schwarz_tau, fp32_bound, df64=df64)
        r = _abi.hf_uhf_result()
        out = {}
        if outputs:
            n = self.nbf
            dev = torch.device("cuda", self.ctx.device)
            for k in ("Da", "Db"):
                out[k] = torch.empty((n, n), dtype=torch.float64, device=dev)
                setattr(r, k, out[k].data_ptr())
            for k in ("eps_a", "eps_b"):
                out[k] = torch.empty((n,), dtype=torch.float64, device=dev)
                setattr(r, k, out[k].data_ptr())
        ok = (_abi.HF_OK, _abi.HF_ERR_NOT_CONVERGED) if allow_unconverged else (_abi.HF_OK,)
        rc = _check(_lib().hf_uhf_solve(self._h, int(n_alpha), int(n_beta), C.byref(o), C.byref(r)),
                    "hf_uhf_solve", ok)
        return UHFResult(rc=rc, energy=r.energy, e_elec=r.e_elec, e_nuc=r.e_nuc, delta_e=r.delta_e,
                         diis_error=r.diis_error, s2=r.s2, iterations=r.iterations, converged=bool(r.converged),
                         fock_builds=r.fock_builds, quartets=r.quartets, seconds=r.seconds, tensors=out)


@dataclass
class UHFResult:
    rc: int
    energy: float
    e_elec: float
    e_nuc: float
    delta_e: float
    diis_error: float
    s2: float
    iterations: int
    converged: bool
    fock_builds: int
    quartets: int
    seconds: float
    tensors: dict


@dataclass
class SCFResult:
    rc: int
    energy: float
    e_elec: float
    e_nuc: float
    delta_e: float
    diis_error: float
    homo_lumo_gap: float
    iterations: int
    converged: bool
    fock_builds: int
    quartets: int
    seconds: float
    tensors: dict


def scf_solve_batch(bases, max_iter=128, e_tol=1e-8, diis_size=8, schwarz_tau=1e-12, fp32_bound=0.0,
                    df64=False):
    """hf_scf_solve_batch over Basis objects sharing one context; returns (results, status)."""
    lib = _lib()
    n = len(bases)
    arr = (C.c_void_p * n)(*[b.handle.value for b in bases])
    o = hf_scf_opts_default()
    o.max_iter = max_iter
    o.e_tol = e_tol
    o.diis_size = diis_size
    o.jk = jk_opts(schwarz_tau, fp32_bound, df64=df64)
    res = (hf_scf_result * n)()
    st = (C.c_int * n)()
    rc = lib.hf_scf_solve_batch(arr, n, C.byref(o), res, st)
    _check(rc, "hf_scf_solve_batch", ok=(_abi.HF_OK, _abi.HF_ERR_NOT_CONVERGED))
    return list(res), list(st)


class Server:
    """hf_server: continuous-batching SCF serving loop on a context."""

    def __init__(self, ctx: Context, max_active: int = 64, queue_capacity: int = 100000, hbm_budget: int = 0,
                 max_iter=128, e_tol=1e-8, diis_size=8, schwarz_tau=1e-12, fp32_bound=0.0, df64=False):
        lib = _lib()
        o = hf_serve_opts()
        lib.hf_serve_opts_default(C.byref(o))
        o.max_active = max_active
        o.queue_capacity = queue_capacity
        o.hbm_budget = hbm_budget
        o.scf.max_iter = max_iter
        o.scf.e_tol = e_tol
        o.scf.diis_size = diis_size
        o.scf.jk = jk_opts(schwarz_tau, fp32_bound, df64=df64)
        self._h = C.c_void_p()
        _check(lib.hf_serve_create(ctx.handle, C.byref(o), C.byref(self._h)), "hf_serve_create")
        self.ctx = ctx

    def submit(self, mol, n_electrons: Optional[int] = None) -> int:
        atoms, shells, exps, coefs = _marshal(mol)
        req = hf_request()
        req.atoms = C.cast(atoms, C.POINTER(hf_atom))
        req.natom = len(atoms)
        req.shells = C.cast(shells, C.POINTER(hf_shell))
        req.nshell = len(shells)
        req.exps = exps.ctypes.data_as(C.POINTER(C.c_double))
        req.coefs = coefs.ctypes.data_as(C.POINTER(C.c_double))
        req.nprim = len(exps)
        req.n_electrons = int(mol.n_electrons if n_electrons is None else n_electrons)
        t = C.c_uint64()
        _check(_lib().hf_serve_submit(self._h, C.byref(req), C.byref(t)), "hf_serve_submit")
        return int(t.value)

    def poll(self, ticket: int):
        r = hf_serve_result()
        rc = _lib().hf_serve_poll(self._h, ticket, C.byref(r))
        if rc == _abi.HF_PENDING:
            return None
        _check(rc, "hf_serve_poll")
        return r

    def cancel(self, ticket: int) -> int:
        return _lib().hf_serve_cancel(self._h, ticket)

    def now(self) -> float:
        return float(_lib().hf_serve_now(self._h))

    def drain(self, timeout_s: float = 600.0):
        return _check(_lib().hf_serve_drain(self._h, timeout_s), "hf_serve_drain")

    def close(self):
        if self._h:
            _lib().hf_serve_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- C-named entry points
# One function per C entry point, same name, argument marshalling only.

def hf_ctx_create(device: int = 0, hbm_budget: int = 0, stream=None) -> Context:
    return Context(device, hbm_budget, stream)


def hf_basis_create(ctx: Context, mol, n_electrons: Optional[int] = None) -> Basis:
    return Basis(ctx, mol, n_electrons)


def hf_schwarz(basis: Basis) -> np.ndarray:
    return basis.schwarz()


def hf_count_quartets(basis: Basis, opts: Optional[hf_jk_opts] = None):
    return basis.count_quartets(opts)


def hf_fock_jk(basis: Basis, D, J=None, K=None, opts: Optional[hf_jk_opts] = None):
    return basis.fock_jk(D, J, K, opts)


def hf_fock_jk_noalloc(basis: Basis, D, J, K, opts: Optional[hf_jk_opts] = None):
    _check(_lib().hf_fock_jk_noalloc(basis.handle, _ptr(D), _ptr(J), _ptr(K), C.byref(opts) if opts else None),
           "hf_fock_jk_noalloc")
    return J, K


def hf_one_electron(basis: Basis):
    return basis.one_electron()


def hf_eri_tensor(basis: Basis):
    return basis.eri_tensor()


def hf_jk_stored(basis: Basis, G, D):
    return basis.jk_stored(G, D)


def hf_scf_solve(basis: Basis, **kw) -> SCFResult:
    return basis.scf(**kw)


def hf_uhf_solve(basis: Basis, n_alpha: int, n_beta: int, **kw) -> UHFResult:
    return basis.uhf(n_alpha, n_beta, **kw)


def hf_fock_jk_uhf(basis: Basis, Da, Db, opts: Optional[hf_jk_opts] = None):
    return basis.fock_jk_uhf(Da, Db, opts)


def hf_mp2_energy(basis: Basis, C_mo, eps, n_occ: int) -> float:
    return basis.mp2_energy(C_mo, eps, n_occ)


def hf_rhf_gradient(basis: Basis, scf_result=None, schwarz_tau: float = 1e-12):
    return basis.gradient(scf_result, schwarz_tau)


def hf_scf_solve_batch(bases, **kw):
    return scf_solve_batch(bases, **kw)


def hf_serve_create(ctx: Context, **kw) -> Server:
    return Server(ctx, **kw)


def hf_serve_submit(server: Server, mol, n_electrons: Optional[int] = None) -> int:
    return server.submit(mol, n_electrons)


def hf_serve_poll(server: Server, ticket: int):
    return server.poll(ticket)


def hf_serve_cancel(server: Server, ticket: int) -> int:
    return server.cancel(ticket)


def hf_serve_drain(server: Server, timeout_s: float = 600.0):
    return server.drain(timeout_s)


def hf_rys_rule(n: int, T: float):
    """Roots u_i and weights w_i (numpy arrays) of the n-point Rys rule at T,
    from the library's table (host only)."""
    import numpy as np
    u = (C.c_double * n)() if n > 0 else (C.c_double * 1)()
    w = (C.c_double * n)() if n > 0 else (C.c_double * 1)()
    _check(_lib().hf_rys_rule(int(n), float(T), u, w), "hf_rys_rule")
    return np.array(u[:n]), np.array(w[:n])
