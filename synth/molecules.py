"""Seeded synthetic molecules (geometry, charges, shells, exponents, raw coefficients).

The paper's benchmark systems (atoms and H2O in 3-21G / cc-pVTZ / cc-pVQZ
basis sets, Fig. 3 and Fig. 4) need basis-library files that are not
available here, so the workloads are synthetic molecules of the same size
range built from the rules below.  Every draw comes from
``numpy.random.default_rng(seed)`` (PCG64) in a fixed order: geometry,
charges, then for each shell its exponents followed by its coefficients.

Coordinates are in bohr, as in the paper's input file (Sec. "Using the
code").  Shell angular momentum l is 0..4 (Cartesian s, p, d, f, g).
Coefficients are raw draws; normalisation (Eq. 1 basis functions with unit
self-overlap) is left to the consumer.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List

import numpy as np


@dataclass
class Molecule:
    """One molecule and its contracted Cartesian Gaussian basis (Eq. 1).

    Arrays:
      Z            int32  [natom]       nuclear charges
      xyz          f64    [natom, 3]    nuclear positions (bohr)
      shell_atom   int32  [nshell]      atom index of each shell centre
      shell_l      int32  [nshell]      angular momentum l = L+M+N
      shell_nprim  int32  [nshell]      primitives in the contraction
      shell_prim   int32  [nshell]      offset of the shell's first primitive
      exps         f64    [nprim]       primitive exponents alpha
      coefs        f64    [nprim]       raw contraction coefficients d
    """

    Z: np.ndarray
    xyz: np.ndarray
    shell_atom: np.ndarray
    shell_l: np.ndarray
    shell_nprim: np.ndarray
    shell_prim: np.ndarray
    exps: np.ndarray
    coefs: np.ndarray
    n_electrons: int
    name: str = ""
    seed: int = -1
    meta: dict = field(default_factory=dict)

    @property
    def natom(self) -> int:
        return int(self.Z.shape[0])

    @property
    def nshell(self) -> int:
        return int(self.shell_l.shape[0])

    @property
    def nbf(self) -> int:
        """Number of Cartesian basis functions: (l+1)(l+2)/2 per shell."""
        l = self.shell_l.astype(np.int64)
        return int(((l + 1) * (l + 2) // 2).sum())

    def copy(self) -> "Molecule":
        return Molecule(self.Z.copy(), self.xyz.copy(), self.shell_atom.copy(),
                        self.shell_l.copy(), self.shell_nprim.copy(),
                        self.shell_prim.copy(), self.exps.copy(),
                        self.coefs.copy(), self.n_electrons, self.name,
                        self.seed, dict(self.meta))


def _pack(Z, xyz, shells, name, seed, n_electrons=None) -> Molecule:
    """shells: list of (atom, l, exps[], coefs[])."""
    sa, sl, sn, sp, ex, co = [], [], [], [], [], []
    off = 0
    for atom, l, e, c in shells:
        sa.append(atom)
        sl.append(l)
        sn.append(len(e))
        sp.append(off)
        ex.extend(float(v) for v in e)
        co.extend(float(v) for v in c)
        off += len(e)
    Z = np.asarray(Z, dtype=np.int32)
    if n_electrons is None:
        n_electrons = int(Z.sum())
        if n_electrons % 2:
            # Closed-shell RHF needs an even count: an odd total is read as
            # the singly charged cation.
            n_electrons -= 1
    return Molecule(Z=Z, xyz=np.asarray(xyz, dtype=np.float64).reshape(-1, 3),
                    shell_atom=np.asarray(sa, dtype=np.int32),
                    shell_l=np.asarray(sl, dtype=np.int32),
                    shell_nprim=np.asarray(sn, dtype=np.int32),
                    shell_prim=np.asarray(sp, dtype=np.int32),
                    exps=np.asarray(ex, dtype=np.float64),
                    coefs=np.asarray(co, dtype=np.float64),
                    n_electrons=int(n_electrons), name=name, seed=seed)


def _log_uniform(rng, lo, hi, n):
    return np.exp(rng.uniform(np.log(lo), np.log(hi), size=n))


def h_line(n_atoms: int = 8, seed: int = 0, spacing: float = 1.4,
           jitter: float = 0.1, nprim: int = 3,
           exp_range=(0.1, 10.0), coef_range=(0.2, 1.0)) -> Molecule:
    """Hydrogen chain on a jittered line, one contracted s shell per atom.

    x_i = spacing*i + U(-jitter, jitter); y, z = U(-jitter, jitter).
    Defaults: 8 atoms, 1.4 bohr, 3 primitives with exponents log-uniform in
    [0.1, 10] and coefficients uniform in [0.2, 1]; 8 electrons.
    """
    rng = np.random.default_rng(seed)
    xyz = np.zeros((n_atoms, 3))
    for i in range(n_atoms):
        d = rng.uniform(-jitter, jitter, size=3)
        xyz[i] = (spacing * i + d[0], d[1], d[2])
    Z = np.ones(n_atoms, dtype=np.int32)
    shells = []
    for a in range(n_atoms):
        e = _log_uniform(rng, *exp_range, nprim)
        c = rng.uniform(*coef_range, size=nprim)
        shells.append((a, 0, e, c))
    return _pack(Z, xyz, shells, f"h_line{n_atoms}_s{seed}", seed)


# Basis rules.  "sp": hydrogen 2 s shells, C/O 3 s + 2 p, 3 primitives each,
# exponents log-uniform in [0.05, 50].  "spd": as "sp" plus one Cartesian d
# shell on C/O, 1..6 primitives per shell, exponents log-uniform [0.03, 200].
BASIS_RULES = {
    "sp": dict(h=[0, 0], heavy=[0, 0, 0, 1, 1], nprim=(3, 3), exp=(0.05, 50.0)),
    "spd": dict(h=[0, 0], heavy=[0, 0, 0, 1, 1, 2], nprim=(1, 6), exp=(0.03, 200.0)),
    "s": dict(h=[0], heavy=[0, 0], nprim=(3, 3), exp=(0.1, 10.0)),
    "spdfg": dict(h=[0, 0, 1], heavy=[0, 0, 0, 1, 1, 2, 3, 4], nprim=(1, 3), exp=(0.1, 30.0)),
}


def lattice_molecule(n_atoms: int, seed: int, rules: str = "sp",
                     spacing: float = 2.4, jitter: float = 0.3,
                     charges=(1, 6, 8), charge_p=(0.5, 0.3, 0.2),
                     coef_range=(0.2, 1.0)) -> Molecule:
    """Atoms on a jittered simple-cubic lattice with a random s/p(/d) basis.

    Sites: the smallest n with n**3 >= n_atoms; the first n_atoms sites in
    lexicographic (i, j, k) order; each coordinate = spacing*index +
    U(-jitter, jitter).  Charges drawn from ``charges`` with ``charge_p``.
    """
    rr = BASIS_RULES[rules]
    rng = np.random.default_rng(seed)
    n = 1
    while n ** 3 < n_atoms:
        n += 1
    sites = [(i, j, k) for i in range(n) for j in range(n) for k in range(n)][:n_atoms]
    xyz = np.zeros((n_atoms, 3))
    for a, s in enumerate(sites):
        xyz[a] = spacing * np.asarray(s, dtype=np.float64) + rng.uniform(-jitter, jitter, size=3)
    Z = rng.choice(np.asarray(charges), size=n_atoms, p=np.asarray(charge_p)).astype(np.int32)
    shells = []
    for a in range(n_atoms):
        ls = rr["h"] if Z[a] == 1 else rr["heavy"]
        for l in ls:
            k = int(rng.integers(rr["nprim"][0], rr["nprim"][1] + 1))
            e = _log_uniform(rng, *rr["exp"], k)
            c = rng.uniform(*coef_range, size=k)
            shells.append((a, l, e, c))
    m = _pack(Z, xyz, shells, f"lattice{n_atoms}_{rules}_s{seed}", seed)
    m.meta["rules"] = rules
    return m


# Shape of a correlation-consistent quadruple-zeta basis, the basis of the
# paper's HF timing benchmark (H2O, Fig. 4): per element, the shells as
# (l, primitives).  O: 5s4p3d2f1g with two s shells contracted over 12
# primitives and one p shell over 6; H: 4s3p2d1f with one s shell over 4.
QZ_SHAPE = {
    8: [(0, 12), (0, 12), (0, 1), (0, 1), (0, 1), (1, 6), (1, 1), (1, 1), (1, 1),
        (2, 1), (2, 1), (2, 1), (3, 1), (3, 1), (4, 1)],
    1: [(0, 4), (0, 1), (0, 1), (0, 1), (1, 1), (1, 1), (1, 1), (2, 1), (2, 1), (3, 1)],
}
# exponent range per element and l (contracted shells draw log-uniform in
# it; the single-primitive shells of one l are even-tempered across it with
# a jitter of 0.2 of a step)
QZ_EXP = {
    8: {0: (0.1, 6.0e4), 1: (0.1, 60.0), 2: (0.3, 4.0), 3: (0.5, 3.0), 4: (1.0, 2.5)},
    1: {0: (0.05, 80.0), 1: (0.2, 3.0), 2: (0.5, 2.5), 3: (0.8, 1.5)},
}


def water_qz(seed: int = 0, coef_range=(0.2, 1.0)) -> Molecule:
    """H2O (O-H 1.809 bohr, H-O-H 104.5 degrees) with a synthetic basis of
    the quadruple-zeta shape above: nbf 140 (Cartesian), 10 electrons."""
    rng = np.random.default_rng(seed)
    half = np.deg2rad(104.5) / 2
    r = 1.809
    xyz = np.array([[0.0, 0.0, 0.0], [r * np.sin(half), r * np.cos(half), 0.0],
                    [-r * np.sin(half), r * np.cos(half), 0.0]])
    Z = [8, 1, 1]
    shells = []
    for a, z in enumerate(Z):
        spec = QZ_SHAPE[z]
        for l in sorted({l for l, _ in spec}):
            lo, hi = QZ_EXP[z][l]
            single = [k for ll, k in spec if ll == l and k == 1]
            for ll, k in spec:
                if ll == l and k > 1:
                    shells.append((a, l, _log_uniform(rng, lo, hi, k), rng.uniform(*coef_range, size=k)))
            ns = len(single)
            for i in range(ns):
                t = (i + 0.5 + rng.uniform(-0.2, 0.2)) / ns
                shells.append((a, l, np.array([lo * (hi / lo) ** t]), np.array([1.0])))
    return _pack(Z, xyz, shells, f"water_qz_s{seed}", seed)


def water_cluster_qz(n: int = 8, seed: int = 0, spacing: float = 5.7) -> Molecule:
    """n copies of water_qz(seed) (same basis on every copy, as a basis set
    is per element) on a simple-cubic lattice of the given spacing (bohr),
    each rotated by a random rotation (QR of a Gaussian 3x3 matrix, drawn
    from default_rng(seed + 1) in molecule order): nbf 140 n, 10 n
    electrons."""
    w = water_qz(seed)
    rng = np.random.default_rng(seed + 1)
    m = 1
    while m ** 3 < n:
        m += 1
    sites = [(i, j, k) for i in range(m) for j in range(m) for k in range(m)][:n]
    Z, xyz, shells = [], [], []
    com = w.xyz.mean(axis=0)
    for c, site in enumerate(sites):
        q, r = np.linalg.qr(rng.normal(size=(3, 3)))
        q = q * np.sign(np.diag(r))
        if np.linalg.det(q) < 0:
            q[:, 0] = -q[:, 0]
        pos = (w.xyz - com) @ q.T + spacing * np.asarray(site, dtype=np.float64)
        for a in range(w.natom):
            Z.append(int(w.Z[a]))
            xyz.append(pos[a])
        for sh in range(w.nshell):
            o, k = int(w.shell_prim[sh]), int(w.shell_nprim[sh])
            shells.append((c * w.natom + int(w.shell_atom[sh]), int(w.shell_l[sh]), w.exps[o:o + k], w.coefs[o:o + k]))
    return _pack(Z, xyz, shells, f"water{n}_qz_s{seed}", seed)


def small_f_molecule(seed: int = 0) -> Molecule:
    """O-H (1.9 bohr) with an f shell on O: O s(3) s(1) p(2) f(1), H s(2)
    s(1) (primitives in parentheses), exponents log-uniform in [0.3, 6],
    coefficients uniform in [0.2, 1]; 8 electrons (the cation)."""
    rng = np.random.default_rng(seed)
    xyz = np.array([[0.0, 0.0, 0.0], [0.0, 0.3, 1.9]])
    spec = [(0, 0, 3), (0, 0, 1), (0, 1, 2), (0, 3, 1), (1, 0, 2), (1, 0, 1)]
    shells = [(a, l, _log_uniform(rng, 0.3, 6.0, k), rng.uniform(0.2, 1.0, size=k)) for a, l, k in spec]
    return _pack([8, 1], xyz, shells, f"small_f_s{seed}", seed)


def small_g_molecule(seed: int = 0) -> Molecule:
    """O-H (1.9 bohr) with a g shell on O and a d shell on H: O s(3) s(1)
    p(2) g(1), H s(2) d(1) (primitives in parentheses), exponents
    log-uniform in [0.3, 6], coefficients uniform in [0.2, 1]; 8 electrons
    (the cation)."""
    rng = np.random.default_rng(seed)
    xyz = np.array([[0.0, 0.0, 0.0], [0.2, 0.1, 1.9]])
    spec = [(0, 0, 3), (0, 0, 1), (0, 1, 2), (0, 4, 1), (1, 0, 2), (1, 2, 1)]
    shells = [(a, l, _log_uniform(rng, 0.3, 6.0, k), rng.uniform(0.2, 1.0, size=k)) for a, l, k in spec]
    return _pack([8, 1], xyz, shells, f"small_g_s{seed}", seed)


def random_shells_molecule(ls, seed: int, nprim=(1, 3), exp_range=(0.2, 3.0),
                           box: float = 1.5, coef_range=(0.2, 1.0),
                           Z=None) -> Molecule:
    """A tiny molecule with one atom per shell of angular momenta ``ls``.

    Used for unit tests on single shell quartets: centres uniform in a cube
    of side ``box`` bohr, exponents log-uniform in ``exp_range``.
    """
    rng = np.random.default_rng(seed)
    na = len(ls)
    xyz = rng.uniform(-box / 2, box / 2, size=(na, 3))
    if Z is None:
        Z = np.ones(na, dtype=np.int32)
    shells = []
    for a, l in enumerate(ls):
        k = int(rng.integers(nprim[0], nprim[1] + 1))
        e = _log_uniform(rng, *exp_range, k)
        c = rng.uniform(*coef_range, size=k)
        shells.append((a, int(l), e, c))
    ne = int(np.sum(Z))
    ne -= ne % 2
    return _pack(Z, xyz, shells, f"shells{''.join(map(str, ls))}_s{seed}", seed,
                 n_electrons=ne)


def batch_molecules(count: int = 512, seed_base: int = 1000, atoms=(4, 60),
                    rules: str = "sp", size_seed: int = 999) -> List[Molecule]:
    """Independent molecules for batched SCF: atom counts uniform in ``atoms``.

    Molecule i uses seed ``seed_base + i``; the atom counts come from their
    own stream seeded with ``size_seed``.
    """
    rng = np.random.default_rng(size_seed)
    sizes = rng.integers(atoms[0], atoms[1] + 1, size=count)
    return [lattice_molecule(int(n), seed_base + i, rules) for i, n in enumerate(sizes)]


def serve_stream(n_requests: int = 20000, rate: float = 200.0, seed: int = 7,
                 mol_seed_base: int = 10000, atoms=(4, 150), rules: str = "spd"):
    """Poisson arrival stream: returns (arrival_times_s, atom_counts, seeds).

    Inter-arrival times are exponential with mean 1/rate; atom counts are
    log-uniform in ``atoms`` (rounded); molecule i is
    ``lattice_molecule(atom_counts[i], seeds[i], rules)``.
    """
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=n_requests)
    t = np.cumsum(gaps)
    sizes = np.rint(np.exp(rng.uniform(np.log(atoms[0]), np.log(atoms[1]), size=n_requests)))
    seeds = mol_seed_base + np.arange(n_requests)
    return t, sizes.astype(np.int64), seeds.astype(np.int64)


def concat_basis(mols: List[Molecule]):
    """Offsets of each molecule inside a packed batch (shells, prims, atoms, bf)."""
    out = []
    so = po = ao = bo = 0
    for m in mols:
        out.append(dict(shell=so, prim=po, atom=ao, bf=bo))
        so += m.nshell
        po += int(m.exps.shape[0])
        ao += m.natom
        bo += m.nbf
    return out


def shell_bf_offsets(mol: Molecule) -> np.ndarray:
    """First basis function of each shell (Cartesian: 1, 3, 6 per s, p, d),
    with a final entry equal to nbf."""
    l = mol.shell_l.astype(np.int64)
    return np.concatenate([[0], np.cumsum((l + 1) * (l + 2) // 2)])


def shell_supported_density(mol: Molecule, seed: int = 11, n_random: int = 4, n_occ: int = 6):
    """A symmetric positive semidefinite density C C^T whose support is a few
    shells: ``n_random`` shells drawn at random plus, when the molecule has d
    shells, its first d shell and the middle one.  Returns (D, shells, rows)
    where ``rows`` = [first and last supported function, 0, nbf//2, nbf-1]
    are the J/K rows a sampled comparison looks at.

    Only the rows of J and K that touch the support need the quartets
    through those shells, which keeps a CPU comparison at several hundred
    basis functions to minutes.
    """
    rng = np.random.default_rng(seed)
    dsh = [s for s in range(mol.nshell) if mol.shell_l[s] == 2]
    pick = rng.choice(mol.nshell, size=n_random, replace=False).tolist()
    if dsh:
        pick += [dsh[0], dsh[len(dsh) // 2]]
    shells = sorted(set(pick))
    off = shell_bf_offsets(mol)
    nbf = int(off[-1])
    idx = np.concatenate([np.arange(off[s], off[s + 1]) for s in shells])
    C = np.zeros((nbf, n_occ))
    C[idx] = rng.normal(size=(idx.size, n_occ)) / np.sqrt(idx.size)
    rows = np.array([int(idx[0]), int(idx[-1]), 0, nbf // 2, nbf - 1])
    return C @ C.T, shells, rows
