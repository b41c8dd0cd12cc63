"""Textbook closed-shell RHF iteration (test infrastructure).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The steps follow the Szabo-Ostlund SCF procedure the paper builds on
(Sec. "Introduction" and "Capabilities": Hartree-Fock; DIIS of Pulay in
Sec. "Technical details"):

1. X = S^{-1/2} (symmetric Loewdin orthogonalisation, X = U s^{-1/2} U^T);
   lambda_min(S) < 1e-10 is rejected as linear dependence.
2. Core guess: D_0 = 0, so F_0 = H = T + V.
3. For k = 1 .. max_iter:
   F' = X^T F_{k-1} X;  F' C' = C' eps (ascending);  C = X C';
   D_k = C_occ C_occ^T with n_occ = N_e / 2;
   J, K from D_k (J/K equation with P = D_k);  F_k = H + 2J - K;
   E_k = Tr[D_k (H + F_k)] + E_nuc;
   with DIIS on: error e_k = F_k D_k S - S D_k F_k, keep the most recent
   ``diis_size`` (F, e); once two or more are stored, replace F_k by
   sum_i c_i F_i with c from the Pulay system [B -1; -1 0][c; lam] = [0; -1],
   B_ij = <e_i, e_j>; when B is singular (cond > 1e14) the oldest pair is
   dropped and the system solved again;
   stop when |E_k - E_{k-1}| <= e_tol.

With P = 2 D this is the same as Szabo-Ostlund's F = H + J[P] - K[P]/2.
The eigen-decompositions and the small linear solve use numpy's LAPACK
routines as plain library steps.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

from .core import Basis


class LinearDependence(ValueError):
    pass


@dataclass
class RHFResult:
    energy: float
    e_elec: float
    e_nuc: float
    converged: bool
    iterations: int
    D: np.ndarray
    C: np.ndarray
    eps: np.ndarray
    F: np.ndarray          # F_k of the last iteration, before any DIIS extrapolation
    F1: np.ndarray         # F_1 = F(D_1), D_1 from diagonalising H
    energies: List[float] = field(default_factory=list)
    homo_lumo_gap: float = float("nan")
    diis_error: float = float("nan")
    H: Optional[np.ndarray] = None
    S: Optional[np.ndarray] = None


def lowdin(S: np.ndarray, min_eig: float = 1e-10) -> np.ndarray:
    """Symmetric (Loewdin) orthogonaliser X = S^(-1/2) = U s^(-1/2) U^T, step 1
    of the Szabo-Ostlund procedure; LinearDependence below min_eig."""
    s, U = np.linalg.eigh(S)
    if s[0] < min_eig:
        raise LinearDependence(f"lambda_min(S) = {s[0]:.3e} < {min_eig:g}")
    return (U * (1.0 / np.sqrt(s))) @ U.T


def diis_extrapolate(Fs, es):
    """Pulay DIIS (named in Sec. "Technical details"): returns sum_i c_i F_i
    with sum_i c_i = 1 minimising |sum c_i e_i|."""
    Fs = list(Fs)
    es = list(es)
    while len(Fs) >= 2:
        m = len(Fs)
        B = np.empty((m + 1, m + 1))
        for i in range(m):
            for j in range(m):
                B[i, j] = float(np.sum(es[i] * es[j]))
        B[m, :m] = -1.0
        B[:m, m] = -1.0
        B[m, m] = 0.0
        rhs = np.zeros(m + 1)
        rhs[m] = -1.0
        if np.linalg.cond(B) > 1e14:
            Fs.pop(0)
            es.pop(0)
            continue
        c = np.linalg.solve(B, rhs)[:m]
        return sum(ci * Fi for ci, Fi in zip(c, Fs))
    return Fs[-1]


def rhf(mol, max_iter: int = 30, e_tol: float = 1e-8, diis_size: int = 0,
        tau: float = 0.0, nthreads: int = 1, basis: Optional[Basis] = None,
        D0: Optional[np.ndarray] = None) -> RHFResult:
    """Closed-shell RHF by the steps of the module docstring (Szabo-Ostlund,
    the procedure the paper's Hartree-Fock follows; J/K from the oracle's
    integrals, optionally Schwarz-screened with its own factors)."""
    B = basis if basis is not None else Basis(mol)
    S, T, V = B.one_electron()
    H = T + V
    e_nuc = B.nuclear_repulsion()
    X = lowdin(S)
    nocc = mol.n_electrons // 2
    if D0 is None:
        F = H.copy()
    else:
        J, K, _ = B.jk(D0, tau, nthreads)
        F = H + 2.0 * J - K
    e_old = None
    energies = []
    Fs, es = [], []
    F1 = None
    converged = False
    k = 0
    for k in range(1, max_iter + 1):
        Fp = X.T @ F @ X
        eps, Cp = np.linalg.eigh(Fp)
        C = X @ Cp
        Cocc = C[:, :nocc]
        D = Cocc @ Cocc.T
        J, K, _ = B.jk(D, tau, nthreads)
        Fk = H + 2.0 * J - K
        E = float(np.sum(D * (H + Fk))) + e_nuc
        energies.append(E)
        if F1 is None:
            F1 = Fk.copy()
        err = Fk @ D @ S - S @ D @ Fk
        F = Fk
        if diis_size > 0:
            Fs.append(Fk)
            es.append(err)
            if len(Fs) > diis_size:
                Fs.pop(0)
                es.pop(0)
            if len(Fs) >= 2:
                F = diis_extrapolate(Fs, es)
        if e_old is not None and abs(E - e_old) <= e_tol:
            converged = True
            break
        e_old = E
    gap = float(eps[nocc] - eps[nocc - 1]) if nocc < eps.shape[0] and nocc > 0 else float("nan")
    return RHFResult(energy=E, e_elec=E - e_nuc, e_nuc=e_nuc, converged=converged,
                     iterations=k, D=D, C=C, eps=eps, F=Fk, F1=F1, energies=energies,
                     homo_lumo_gap=gap, diis_error=float(np.abs(err).max()), H=H, S=S)


@dataclass
class UHFResult:
    energy: float
    e_nuc: float
    converged: bool
    iterations: int
    Da: np.ndarray
    Db: np.ndarray
    Ca: np.ndarray
    Cb: np.ndarray
    eps_a: np.ndarray
    eps_b: np.ndarray
    s2: float               # <S^2> of the UHF determinant
    energies: List[float] = field(default_factory=list)


def uhf(mol, n_alpha: int, n_beta: int, max_iter: int = 128, e_tol: float = 1e-8, diis_size: int = 0,
        tau: float = 0.0, nthreads: int = 1, basis: Optional[Basis] = None) -> UHFResult:
    """Unrestricted HF (the paper's test calculations are UHF), by the
    Pople-Nesbet equations as Szabo-Ostlund state them:

      D^s = C^s_occ C^s_occ^T (s = alpha, beta; n_alpha and n_beta columns),
      F^s = H + J[D^a + D^b] - K[D^s]   (J, K of the J/K equation, no factors),
      E = (1/2) sum_s Tr[D^s (H + F^s)] + E_nuc,

    X = S^(-1/2), core guess F^a = F^b = H, stop at |E_k - E_{k-1}| <= e_tol.
    With DIIS the alpha and beta errors e^s = F^s D^s S - S D^s F^s form one
    vector and share one set of coefficients.  <S^2> = S_z (S_z + 1) + n_beta
    - sum_ij |(C^a_occ^T S C^b_occ)_ij|^2 with S_z = (n_alpha - n_beta) / 2."""
    B = basis if basis is not None else Basis(mol)
    S, T, V = B.one_electron()
    H = T + V
    e_nuc = B.nuclear_repulsion()
    X = lowdin(S)
    nocc = (n_alpha, n_beta)
    F = [H.copy(), H.copy()]
    e_old = None
    energies = []
    Fs, es = [], []
    converged = False
    k = 0
    for k in range(1, max_iter + 1):
        Cs, epss, Ds = [], [], []
        for s in range(2):
            eps, Cp = np.linalg.eigh(X.T @ F[s] @ X)
            C = X @ Cp
            Cs.append(C)
            epss.append(eps)
            Ds.append(C[:, :nocc[s]] @ C[:, :nocc[s]].T)
        Ja, Ka, _ = B.jk(Ds[0], tau, nthreads)
        Jb, Kb, _ = B.jk(Ds[1], tau, nthreads)
        J = Ja + Jb                        # J is linear in D
        Fk = [H + J - Ka, H + J - Kb]
        E = 0.5 * sum(float(np.sum(Ds[s] * (H + Fk[s]))) for s in range(2)) + e_nuc
        energies.append(E)
        F = Fk
        if diis_size > 0:
            Fs.append(np.stack(Fk))
            es.append(np.stack([Fk[s] @ Ds[s] @ S - S @ Ds[s] @ Fk[s] for s in range(2)]))
            if len(Fs) > diis_size:
                Fs.pop(0)
                es.pop(0)
            if len(Fs) >= 2:
                Fx = diis_extrapolate(Fs, es)
                F = [Fx[0], Fx[1]]
        if e_old is not None and abs(E - e_old) <= e_tol:
            converged = True
            break
        e_old = E
    sz = 0.5 * (n_alpha - n_beta)
    ov = Cs[0][:, :n_alpha].T @ S @ Cs[1][:, :n_beta]
    s2 = sz * (sz + 1.0) + n_beta - float(np.sum(ov * ov))
    return UHFResult(energy=E, e_nuc=e_nuc, converged=converged, iterations=k, Da=Ds[0], Db=Ds[1],
                     Ca=Cs[0], Cb=Cs[1], eps_a=epss[0], eps_b=epss[1], s2=s2, energies=energies)


def mp2(result: RHFResult, basis: Basis, n_occ: int) -> float:
    """Second-order Moller-Plesset correlation energy of a converged
    closed-shell RHF solution (the paper's MP2 follows Szabo-Ostlund):

      E(2) = sum_{i,j occ} sum_{a,b virt} (ia|jb) [2 (ia|jb) - (ib|ja)]
                                           / (e_i + e_j - e_a - e_b)

    over the canonical spatial orbitals, (ia|jb) in chemists' notation from
    the AO tensor by four one-index transformations (numpy contractions as
    library steps).  Small bases only: it builds the N^4 AO tensor."""
    G = basis.eri_tensor()
    C, eps = result.C, result.eps
    Co, Cv = C[:, :n_occ], C[:, n_occ:]
    t = np.einsum("pqrs,pi->iqrs", G, Co)
    t = np.einsum("iqrs,qa->iars", t, Cv)
    t = np.einsum("iars,rj->iajs", t, Co)
    iajb = np.einsum("iajs,sb->iajb", t, Cv)
    eo, ev = eps[:n_occ], eps[n_occ:]
    denom = eo[:, None, None, None] - ev[None, :, None, None] + eo[None, None, :, None] - ev[None, None, None, :]
    return float(np.sum(iajb * (2.0 * iajb - iajb.transpose(0, 3, 2, 1)) / denom))


def rhf_gradient(mol, h: float = 2e-3, e_tol: float = 1e-13, diis_size: int = 8, max_iter: int = 200) -> np.ndarray:
    """Nuclear gradient dE/dR_A (natom x 3, Eh/bohr) of the converged RHF
    energy; the force on atom A (the paper's HF forces) is its negative.

    By its definition, the derivative of E with the basis functions moving
    with their atoms: central differences at steps h and h/2 combined by
    Richardson extrapolation, g = (4 g(h/2) - g(h)) / 3, error O(h^4).  Each
    displaced SCF starts from the reference density so it converges to the
    same state."""
    ref = rhf(mol, max_iter=max_iter, e_tol=e_tol, diis_size=diis_size)
    if not ref.converged:
        raise RuntimeError("reference SCF did not converge")

    def energy(a, x, d):
        m = mol.copy()
        m.xyz[a, x] += d
        r = rhf(m, max_iter=max_iter, e_tol=e_tol, diis_size=diis_size, D0=ref.D)
        if not r.converged:
            raise RuntimeError("displaced SCF did not converge")
        return r.energy

    g = np.zeros((mol.natom, 3))
    for a in range(mol.natom):
        for x in range(3):
            gh = (energy(a, x, h) - energy(a, x, -h)) / (2 * h)
            gh2 = (energy(a, x, h / 2) - energy(a, x, -h / 2)) / h
            g[a, x] = (4 * gh2 - gh) / 3
    return g
