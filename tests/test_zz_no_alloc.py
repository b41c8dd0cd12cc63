"""hf_fock_jk_noalloc: the J/K build for callers that cannot allocate device
memory (a frozen allocator, a framework that owns all device memory, a
real-time loop).  It keeps its scratch in a static device array of the
library, so its results must equal those of hf_fock_jk, call after call,
even though every call reuses the same scratch.

Collected last (file name) so that a run stopping at the first failure has
run every other test first; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

JK_TOL = 1e-10   # the tolerance the J/K parity tests use


@pytest.fixture(scope="module")
def hf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1303_4916_gb300 as hf
    return hf


def _density(n, seed, nocc):
    rng = np.random.default_rng(seed)
    C = rng.normal(size=(n, nocc)) / np.sqrt(n)
    return C @ C.T


# every precision tier of hf_fock_jk: plain FP64, the FP32 split (with the
# Boys function in FP64 or FP32) and the df64 tier.  The no-alloc call runs
# the same kernels on the same work lists, so in every tier it differs from
# hf_fock_jk only by the order of the FP64 atomic additions.
TIERS = {
    "fp64": {},
    "fp32_split": {"fp32_bound": 1e-5},
    "fp32_split_fp32boys": {"fp32_bound": 1e-5, "fp32_boys": True},
    "df64": {"df64": True},
    "fp32_split_df64": {"fp32_bound": 1e-5, "df64": True},
}


@pytest.mark.parametrize("tier", sorted(TIERS))
@pytest.mark.parametrize("natom,seed,rules", [(8, 12, "sp"), (5, 3, "spd")])
def test_noalloc_matches_fock_jk_on_two_calls(hf, natom, seed, rules, tier):
    import torch
    from synth import lattice_molecule
    lib = hf.load()
    ctx = hf.Context(0)
    basis = hf.Basis(ctx, lattice_molecule(natom, seed, rules))
    n = basis.nbf
    opts = hf.jk_opts(**TIERS[tier])
    D = torch.tensor(_density(n, seed, max(1, basis.n_electrons // 2)), dtype=torch.float64, device="cuda:0")
    J0, K0 = basis.fock_jk(D, opts=opts)          # reference; also builds the work lists
    for call in range(2):
        J = torch.full_like(D, float("nan"))
        K = torch.full_like(D, float("nan"))
        rc = lib.hf_fock_jk_noalloc(basis.handle, D.data_ptr(), J.data_ptr(), K.data_ptr(), ctypes.byref(opts))
        assert rc == 0, lib.hf_last_error()
        torch.cuda.synchronize()
        assert float((J - J0).abs().max()) <= JK_TOL, (tier, call)
        assert float((K - K0).abs().max()) <= JK_TOL, (tier, call)
        D = D * 0.5                                # second call: different density, same scratch
        J0, K0 = basis.fock_jk(D, opts=opts)


def test_noalloc_df64_is_the_df64_tier(hf):
    """With HF_JK_DF64 the no-alloc call runs the df64 kernels, not the FP64
    ones: its result sits on hf_fock_jk's df64 result (atomic-order noise)
    and measurably away from the FP64 result (the tiers round differently)."""
    import torch
    from synth import lattice_molecule
    lib = hf.load()
    ctx = hf.Context(0)
    basis = hf.Basis(ctx, lattice_molecule(5, 3, "spd"))
    n = basis.nbf
    D = torch.tensor(_density(n, 3, max(1, basis.n_electrons // 2)), dtype=torch.float64, device="cuda:0")
    odf = hf.jk_opts(df64=True)
    J64, K64 = basis.fock_jk(D, opts=hf.jk_opts())
    Jdf, Kdf = basis.fock_jk(D, opts=odf)
    J = torch.empty_like(D)
    K = torch.empty_like(D)
    rc = lib.hf_fock_jk_noalloc(basis.handle, D.data_ptr(), J.data_ptr(), K.data_ptr(), ctypes.byref(odf))
    assert rc == 0, lib.hf_last_error()
    torch.cuda.synchronize()
    dist = lambda a, b: float((a - b).abs().max())
    d_tiers = max(dist(Jdf, J64), dist(Kdf, K64))
    d_same = max(dist(J, Jdf), dist(K, Kdf))
    assert d_same <= JK_TOL and d_tiers <= JK_TOL
    if d_tiers < 1e-13:
        pytest.skip(f"the tiers agree to {d_tiers:.1e} on this molecule")
    assert d_same < 0.25 * d_tiers, (d_same, d_tiers)


def test_noalloc_rejects_what_it_cannot_serve(hf):
    import torch
    from synth import lattice_molecule
    lib = hf.load()
    ctx = hf.Context(0)
    small = hf.Basis(ctx, lattice_molecule(3, 1, "sp"))
    D = torch.zeros((small.nbf, small.nbf), dtype=torch.float64, device="cuda:0")
    J = torch.empty_like(D)
    K = torch.empty_like(D)
    other = hf.jk_opts(schwarz_tau=1e-9)         # no work lists prepared for these options
    rc = lib.hf_fock_jk_noalloc(small.handle, D.data_ptr(), J.data_ptr(), K.data_ptr(), ctypes.byref(other))
    assert rc == -1 and b"work lists" in lib.hf_last_error()
    bad = hf.jk_opts(schwarz_tau=-1.0)           # thresholds are checked before the work lists
    rc = lib.hf_fock_jk_noalloc(small.handle, D.data_ptr(), J.data_ptr(), K.data_ptr(), ctypes.byref(bad))
    assert rc == -1 and b"negative threshold" in lib.hf_last_error()
    big = hf.Basis(ctx, lattice_molecule(110, 2, "sp"))   # nbf > 512
    assert big.nbf > 512
    Db = torch.zeros((big.nbf, big.nbf), dtype=torch.float64, device="cuda:0")
    rc = lib.hf_fock_jk_noalloc(big.handle, Db.data_ptr(), Db.data_ptr(), Db.data_ptr(), None)
    assert rc == -12 and b"512" in lib.hf_last_error()
