"""The bounds-checked build (-DHF_BOUNDS_CHECK), the stand-in for a device
memory checker: every work-item, shell-pair, primitive-record and matrix
index of the J/K kernels is tested before use and a failure comes back as an
error naming the index.  Built on the GPU host, run in a child process on
small cases of every angular class (RHF and unrestricted J/K, FP64, df64 and
the FP32 split, single- and multi-molecule launches, the Rys route of the f
and g shells, the gradient), checked against the oracle: no check may fail
and the results are those of the normal build."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
import oracle
import paper_1303_4916_gb300 as hf
from synth import lattice_molecule
lib = hf.load()
out = {"checked": lib.hf_bounds_checked(), "cases": []}
ctx = hf.Context(0)
for natom, seed in ((3, 41), (5, 3)):
    mol = lattice_molecule(natom, seed, "spd")
    b = hf.Basis(ctx, mol)
    ob = oracle.Basis(mol)
    n = b.nbf
    rng = np.random.default_rng(seed)
    Cm = rng.normal(size=(n, 3)) / np.sqrt(n)
    Dn = Cm @ Cm.T
    Jr, Kr, _ = ob.jk(Dn, tau=1e-12, nthreads=oracle.oracle_threads())
    D = torch.tensor(Dn, device="cuda:0")
    for tier in ({}, {"df64": True}, {"fp32_bound": 1e-5}):
        J, K = b.fock_jk(D, opts=hf.jk_opts(**tier))
        torch.cuda.synchronize()
        out["cases"].append([natom, str(tier), float(np.abs(J.cpu().numpy() - Jr).max()),
                             float(np.abs(K.cpu().numpy() - Kr).max())])
    J, Ka, Kb = b.fock_jk_uhf(D, D * 0.5)
    out["cases"].append([natom, "uhf", float(np.abs(J.cpu().numpy() - 1.5 * Jr).max()),
                         float(np.abs(Kb.cpu().numpy() - 0.5 * Kr).max())])
# f and g shells: the Rys kernels (warp and thread forms), their Rys route
# for every class, the unrestricted digestion and the gradient kernels
from synth import random_shells_molecule, small_f_molecule
mol = random_shells_molecule((4, 3, 1, 0), 61, nprim=(1, 2), exp_range=(0.2, 5.0), box=3.0)
b = hf.Basis(ctx, mol)
ob = oracle.Basis(mol)
n = b.nbf
rng = np.random.default_rng(61)
Cm = rng.normal(size=(n, 4)) / np.sqrt(n)
Dn = Cm @ Cm.T
Jr, Kr, _ = ob.jk(Dn, tau=1e-12, nthreads=oracle.oracle_threads())
D = torch.tensor(Dn, device="cuda:0")
for tier in ({}, {"rys": True}):
    J, K = b.fock_jk(D, opts=hf.jk_opts(**tier))
    out["cases"].append(["fg", str(tier), float(np.abs(J.cpu().numpy() - Jr).max()),
                         float(np.abs(K.cpu().numpy() - Kr).max())])
J, Ka, Kb = b.fock_jk_uhf(D, D * 0.5)
out["cases"].append(["fg", "uhf", float(np.abs(J.cpu().numpy() - 1.5 * Jr).max()),
                     float(np.abs(Kb.cpu().numpy() - 0.5 * Kr).max())])
gm = small_f_molecule(0)
gb = hf.Basis(ctx, gm)
gr = gb.scf(max_iter=200, e_tol=1e-12, diis_size=8, schwarz_tau=0.0)
g = gb.gradient(gr, schwarz_tau=0.0)
g0 = np.asarray(json.load(open(sys.argv[1] + "/tests/golden/gradients.json"))["cases"]["small_f"]["gradient"])
out["grad_err"] = float(np.abs(g - g0).max())
mols = [lattice_molecule(3, 51, "sp"), lattice_molecule(2, 101, "spd")]
res, st = hf.scf_solve_batch([hf.Basis(ctx, m) for m in mols], max_iter=64, e_tol=1e-9)
out["batch"] = [float(r.energy) for r in res]
out["batch_ref"] = [float(oracle.rhf(m, max_iter=64, e_tol=1e-9, diis_size=8, tau=1e-12,
                                     nthreads=oracle.oracle_threads()).energy) for m in mols]
print(json.dumps(out))
"""


def test_bounds_checked_build_on_small_cases():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1303_4916_gb300 import build
    lib = build.build_bounds_checked()
    env = dict(os.environ, HF_LIB=lib)
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["checked"] == 1
    for natom, tier, dj, dk in out["cases"]:
        tol = 1e-7 if "fp32_bound" in tier else 1e-10
        assert dj <= tol and dk <= tol, (natom, tier, dj, dk)
    for e, e_ref in zip(out["batch"], out["batch_ref"]):
        assert abs(e - e_ref) <= 1e-8
    assert out["grad_err"] <= 1e-6
