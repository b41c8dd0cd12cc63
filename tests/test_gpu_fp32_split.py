"""The FP32 precision split against a tolerance derived from its bound.

A shell quartet (AB|CD) runs in FP32 when tau <= Q_AB Q_CD < beta (beta =
fp32_bound).  Each of its integrals obeys |(ab|cd)| <= Q_AB Q_CD (Schwarz),
so if the FP32 evaluation and digestion err by at most eps h_AB h_CD
relative to that bound, the FP32 quartets move the J/K equation's sums by at
most

  |dJ_ab| <= eps * sum_{C,D: FP32} h_AB h_CD Q_AB Q_CD sum_{c in C, d in D} |D_cd|
  |dK_ac| <= eps * sum_{B,D: FP32} h_AB h_CD Q_AB Q_CD sum_{b in B, d in D} |D_bd|

(all shell pairs, both orders: J = sum_cd (ab|cd) D_cd over every c, d).
eps = 2^-16 + 36 * 2^-24: FP32 unit roundoff 2^-24 with a growth budget of
2^8 for the vertical recurrence and its cancellations, plus the rounding of an
FP32 digestion sum of at most 36 products; h_AB = (1 + |A - B|)^min(l_A, l_B),
the growth through the horizontal recurrence, whose steps multiply by A - B.
The FP64 build is the reference."""
import numpy as np
import pytest

from synth import lattice_molecule
from synth.molecules import shell_bf_offsets

pytestmark = pytest.mark.gpu
EPS = 2.0 ** -16 + 36 * 2.0 ** -24
TAU, BETA = 1e-12, 1e-5


@pytest.fixture(scope="module")
def hf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1303_4916_gb300 as hf
    return hf


def _bounds(Q, D, off, mol):
    ns = Q.shape[0]
    Dabs = np.zeros((ns, ns))
    for c in range(ns):
        for d in range(ns):
            Dabs[c, d] = np.abs(D[off[c]:off[c + 1], off[d]:off[d + 1]]).sum()
    # the horizontal recurrence moves angular momentum onto the lower-l shell
    # of a pair with a factor A - B per step: rounding grows by up to
    # (1 + |AB|)^min(l_A, l_B) on each side of the quartet
    xyz = np.asarray(mol.xyz)[np.asarray(mol.shell_atom)]
    l = np.asarray(mol.shell_l)
    dist = np.linalg.norm(xyz[:, None, :] - xyz[None, :, :], axis=-1)
    hrr = (1.0 + dist) ** np.minimum(l[:, None], l[None, :])
    P = Q[:, :, None, None] * Q[None, None, :, :]            # P[A,B,C,D] = Q_AB Q_CD
    W = np.where((P >= TAU) & (P < BETA), P * hrr[:, :, None, None] * hrr[None, None, :, :], 0.0)
    tJ = EPS * np.einsum("abcd,cd->ab", W, Dabs)              # per shell pair (A, B)
    tK = EPS * np.einsum("abcd,bd->ac", W, Dabs)              # per shell pair (A, C)
    expand = lambda t: np.repeat(np.repeat(t, np.diff(off), axis=0), np.diff(off), axis=1)
    return expand(tJ), expand(tK)


@pytest.mark.parametrize("natom,seed,rules", [(8, 61, "spd"), (12, 62, "sp")])
def test_fp32_split_within_derived_bound(hf, natom, seed, rules):
    import torch
    mol = lattice_molecule(natom, seed, rules)
    ctx = hf.Context(0)
    b = hf.Basis(ctx, mol)
    n = b.nbf
    rng = np.random.default_rng(seed)
    Cm = rng.normal(size=(n, max(1, mol.n_electrons // 2))) / np.sqrt(n)
    Dn = Cm @ Cm.T
    D = torch.tensor(Dn, device="cuda:0")
    nq, nf = b.count_quartets(hf.jk_opts(schwarz_tau=TAU, fp32_bound=BETA))
    assert nf >= 1000                                         # the split is exercised
    J64, K64 = b.fock_jk(D, opts=hf.jk_opts(schwarz_tau=TAU))
    off = shell_bf_offsets(mol)
    tJ, tK = _bounds(b.schwarz(), Dn, off, mol)
    for tier in ({}, {"df64": True}, {"fp32_boys": True}):
        J, K = b.fock_jk(D, opts=hf.jk_opts(schwarz_tau=TAU, fp32_bound=BETA, **tier))
        dJ = np.abs(J.cpu().numpy() - J64.cpu().numpy())
        dK = np.abs(K.cpu().numpy() - K64.cpu().numpy())
        # the df64 tier's own error (~1e-14 relative) rides on top of the bound
        slack = 1e-11 if tier.get("df64") else 1e-13
        rJ, rK = float((dJ / (tJ + slack)).max()), float((dK / (tK + slack)).max())
        assert rJ <= 1.0 and rK <= 1.0, (tier, rJ, rK)   # largest error / bound
