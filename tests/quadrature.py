"""Brute-force numerical quadrature of Gaussian integrals (pins for the oracle).

This route shares nothing with the oracle's formulas: no Boys function, no
Hermite or Obara-Saika recurrence, no binomial expansion.

* Contracted functions are built from raw primitives: each primitive is
  normalised by its numerically integrated self-overlap, the contraction
  is then normalised the same way (Eq. 1 functions with unit norm).
* 1D integrals of polynomial x Gaussian use Gauss-Hermite nodes after
  completing the square, which is exact for the polynomial degrees here.
* The Coulomb operator uses 1/r = (2/sqrt(pi)) int_0^inf exp(-u^2 r^2) du.
  For fixed u the two-electron integrand is a product over axes of 2D
  Gaussian integrals exp(-x^T M x + 2 b^T x); each is evaluated exactly by
  a Cholesky change of variables and tensor Gauss-Hermite.  The u integral
  is mapped to t in [0, 1) by u = t / (1 - t) and done by Gauss-Legendre.
"""
from __future__ import annotations

import numpy as np

_GH_X, _GH_W = np.polynomial.hermite.hermgauss(12)
_GL_T, _GL_W = np.polynomial.legendre.leggauss(400)
_GL_T = 0.5 * (_GL_T + 1.0)
_GL_W = 0.5 * _GL_W
_U = _GL_T / (1.0 - _GL_T)
_DU = _GL_W / (1.0 - _GL_T) ** 2


def cart_list(l):
    out = []
    for x in range(l, -1, -1):
        for y in range(l - x, -1, -1):
            out.append((x, y, l - x - y))
    return out


def _overlap_1d(la, A, a, lb, B, b):
    """int (x-A)^la (x-B)^lb exp(-a(x-A)^2 - b(x-B)^2) dx by Gauss-Hermite."""
    p = a + b
    P = (a * A + b * B) / p
    c = a * A * A + b * B * B - p * P * P
    x = P + _GH_X / np.sqrt(p)
    f = (x - A) ** la * (x - B) ** lb
    return np.exp(-c) * np.sum(_GH_W * f) / np.sqrt(p)


def _second_deriv_terms(l, b):
    """d^2/dw^2 [w^l e^{-b w^2}] = sum coef * w^power e^{-b w^2}."""
    terms = []
    if l >= 2:
        terms.append((l * (l - 1), l - 2))
    terms.append((-2.0 * b * (2 * l + 1), l))
    terms.append((4.0 * b * b, l + 2))
    return terms


class QuadBasis:
    """Contracted Cartesian functions of a synth.Molecule, normalised numerically."""

    def __init__(self, mol):
        self.funcs = []   # list of (centre[3], powers(3), [(alpha, coef)])
        for s in range(mol.nshell):
            A = mol.xyz[mol.shell_atom[s]]
            l = int(mol.shell_l[s])
            p0, K = int(mol.shell_prim[s]), int(mol.shell_nprim[s])
            for pw in cart_list(l):
                prims = []
                for k in range(K):
                    a = mol.exps[p0 + k]
                    self_ov = np.prod([_overlap_1d(pw[x], 0.0, a, pw[x], 0.0, a) for x in range(3)])
                    prims.append((a, mol.coefs[p0 + k] / np.sqrt(self_ov)))
                f = (np.asarray(A, dtype=np.float64), pw, prims)
                n2 = self._overlap_raw(f, f)
                prims = [(a, c / np.sqrt(n2)) for a, c in prims]
                self.funcs.append((f[0], pw, prims))
        self.mol = mol

    @staticmethod
    def _overlap_raw(f, g):
        A, pa, fa = f
        B, pb, fb = g
        s = 0.0
        for a, ca in fa:
            for b, cb in fb:
                s += ca * cb * np.prod([_overlap_1d(pa[x], A[x], a, pb[x], B[x], b) for x in range(3)])
        return s

    def overlap(self, i, j):
        return self._overlap_raw(self.funcs[i], self.funcs[j])

    def kinetic(self, i, j):
        A, pa, fa = self.funcs[i]
        B, pb, fb = self.funcs[j]
        t = 0.0
        for a, ca in fa:
            for b, cb in fb:
                s1 = [_overlap_1d(pa[x], A[x], a, pb[x], B[x], b) for x in range(3)]
                lap = 0.0
                for x in range(3):
                    d2 = sum(c * _overlap_1d(pa[x], A[x], a, pw, B[x], b)
                             for c, pw in _second_deriv_terms(pb[x], b))
                    others = np.prod([s1[y] for y in range(3) if y != x])
                    lap += d2 * others
                t += ca * cb * (-0.5) * lap
        return t

    def nuclear(self, i, j):
        """-sum_C Z_C <i| 1/|r - C| |j> via the u-transform of 1/r."""
        A, pa, fa = self.funcs[i]
        B, pb, fb = self.funcs[j]
        mol = self.mol
        v = 0.0
        for at in range(mol.natom):
            Cc = mol.xyz[at]
            acc = 0.0
            for a, ca in fa:
                for b, cb in fb:
                    prod = np.ones_like(_U)
                    for x in range(3):
                        prod *= self._axis_1d_u(pa[x], A[x], a, pb[x], B[x], b, Cc[x])
                    acc += ca * cb * (2.0 / np.sqrt(np.pi)) * np.sum(_DU * prod)
            v -= mol.Z[at] * acc
        return v

    @staticmethod
    def _axis_1d_u(la, A, a, lb, B, b, C):
        """For every u node: int (x-A)^la (x-B)^lb e^{-a(x-A)^2 - b(x-B)^2 - u^2 (x-C)^2} dx."""
        u2 = _U ** 2
        p = a + b + u2
        P = (a * A + b * B + u2 * C) / p
        c = a * A * A + b * B * B + u2 * C * C - p * P * P
        x = P[:, None] + _GH_X[None, :] / np.sqrt(p)[:, None]
        f = (x - A) ** la * (x - B) ** lb
        return np.exp(-c) * np.sum(_GH_W[None, :] * f, axis=1) / np.sqrt(p)

    @staticmethod
    def _axis_2d_u(l1, A, a, l2, B, b, l3, Cc, c, l4, D, d):
        """For every u node: the 2D integral over (x1, x2) of
        (x1-A)^l1 (x1-B)^l2 (x2-C)^l3 (x2-D)^l4 exp(-a(x1-A)^2 - b(x1-B)^2
        - c(x2-C)^2 - d(x2-D)^2 - u^2 (x1-x2)^2)."""
        u2 = _U ** 2
        m11 = a + b + u2
        m22 = c + d + u2
        m12 = -u2
        b1 = a * A + b * B
        b2 = c * Cc + d * D
        c0 = a * A * A + b * B * B + c * Cc * Cc + d * D * D
        det = m11 * m22 - m12 * m12
        x01 = (m22 * b1 - m12 * b2) / det
        x02 = (m11 * b2 - m12 * b1) / det
        const = b1 * x01 + b2 * x02 - c0
        # Cholesky M = L L^T, L = [[l11, 0], [l21, l22]]
        l11 = np.sqrt(m11)
        l21 = m12 / l11
        l22 = np.sqrt(m22 - l21 * l21)
        # x = x0 + L^{-T} y ;  L^{-T} = [[1/l11, -l21/(l11 l22)], [0, 1/l22]]
        y1 = _GH_X[None, :, None]
        y2 = _GH_X[None, None, :]
        X1 = x01[:, None, None] + y1 / l11[:, None, None] - (l21 / (l11 * l22))[:, None, None] * y2
        X2 = x02[:, None, None] + y2 / l22[:, None, None]
        f = (X1 - A) ** l1 * (X1 - B) ** l2 * (X2 - Cc) ** l3 * (X2 - D) ** l4
        w = _GH_W[None, :, None] * _GH_W[None, None, :]
        return np.exp(const) * np.sum(w * f, axis=(1, 2)) / (l11 * l22)

    def eri(self, i, j, k, l):
        fs = [self.funcs[q] for q in (i, j, k, l)]
        (A, pa, fa), (B, pb, fb), (Cc, pc, fc), (D, pd, fd) = fs
        tot = 0.0
        for a, ca in fa:
            for b, cb in fb:
                for c, cc in fc:
                    for d, cd in fd:
                        prod = np.ones_like(_U)
                        for x in range(3):
                            prod *= self._axis_2d_u(pa[x], A[x], a, pb[x], B[x], b,
                                                    pc[x], Cc[x], c, pd[x], D[x], d)
                        tot += ca * cb * cc * cd * (2.0 / np.sqrt(np.pi)) * np.sum(_DU * prod)
        return tot
