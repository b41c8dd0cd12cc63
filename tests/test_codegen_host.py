"""The generated per-class recurrence code of the CUDA path
(paper_1303_4916_gb300/csrc/eri_classes.cuh), built for the host by
tests/gen_host_harness.cpp, against recursions written out in this file:

* VRR, all 21 classes: [e0|f0]^(0) from B_m = [00|00]^(m) by the
  Obara-Saika relations in Head-Gordon-Pople form (lowering e before f here;
  the generator lowers f first and picks the axis of largest power);
* HRR, all 21 classes: (a, b+1_i| = (a+1_i, b| + AB_i (a, b| on the bra and
  the same with CD on the ket (lowering along the first non-zero axis here).

Random values stand in for the per-primitive-quartet quantities: both
recurrences are polynomial identities in them, so agreement to rounding
means the generated code is the recurrence.
"""
import ctypes
import importlib.util
import os
import random
import shutil
import subprocess
from functools import lru_cache

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1303_4916_gb300", "csrc")


@pytest.fixture(scope="module")
def gen():
    spec = importlib.util.spec_from_file_location("gen_eri", os.path.join(CSRC, "gen_eri.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    cxx = shutil.which("g++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    out = str(tmp_path_factory.mktemp("gen") / "libgen.so")
    subprocess.run([cxx, "-O1", "-std=c++17", "-shared", "-fPIC", "-Wno-unknown-pragmas", "-I", CSRC,
                    os.path.join(ROOT, "tests", "gen_host_harness.cpp"), "-o", out], check=True)
    return ctypes.CDLL(out)


def _lower(v, i):
    return tuple(x - (k == i) for k, x in enumerate(v))


def _raise(v, i):
    return tuple(x + (k == i) for k, x in enumerate(v))


def _vrr_reference(q, B):
    @lru_cache(maxsize=None)
    def val(e, f, m):
        if sum(e) == 0 and sum(f) == 0:
            return B[m]
        if sum(e) > 0:
            i = next(k for k in range(3) if e[k] > 0)
            e1 = _lower(e, i)
            r = q["PA"][i] * val(e1, f, m) + q["WP"][i] * val(e1, f, m + 1)
            if e1[i] > 0:
                e2 = _lower(e1, i)
                r += e1[i] * q["o2p"] * (val(e2, f, m) - q["rp"] * val(e2, f, m + 1))
            if f[i] > 0:
                r += f[i] * q["o2pq"] * val(e1, _lower(f, i), m + 1)
            return r
        i = next(k for k in range(3) if f[k] > 0)
        f1 = _lower(f, i)
        r = q["QC"][i] * val(e, f1, m) + q["WQ"][i] * val(e, f1, m + 1)
        if f1[i] > 0:
            f2 = _lower(f1, i)
            r += f1[i] * q["o2q"] * (val(e, f2, m) - q["rq"] * val(e, f2, m + 1))
        return r
    return val


def _classes(gen):
    _, cls = gen.classes(2)
    return [(f"C_{gen.LNAME[a]}{gen.LNAME[b]}_{gen.LNAME[c]}{gen.LNAME[d]}", (a, b, c, d)) for a, b, c, d in cls]


def test_generated_vrr_is_the_recurrence(gen, lib):
    rng = random.Random(7)
    classes = _classes(gen)
    assert len(classes) == 21
    for name, (la, lb, lc, ld) in classes:
        L = la + lb + lc + ld
        E, F = gen.Range(la, la + lb), gen.Range(lc, lc + ld)
        q = {n: [rng.uniform(-1, 1) for _ in range(3)] for n in ("PA", "WP", "QC", "WQ")}
        q.update(o2p=rng.uniform(0.05, 2), o2q=rng.uniform(0.05, 2), o2pq=rng.uniform(0.05, 1),
                 rp=rng.uniform(0.1, 0.9), rq=rng.uniform(0.1, 0.9))
        B = [rng.uniform(0.1, 1.0) for _ in range(L + 1)]
        qv = np.array(q["PA"] + q["WP"] + q["QC"] + q["WQ"] + [q["o2p"], q["o2q"], q["o2pq"], q["rp"], q["rq"]])
        acc = np.zeros(len(E) * len(F))
        Bv = np.array(B)
        getattr(lib, f"vrr_{name}")(acc.ctypes.data_as(ctypes.c_void_p), Bv.ctypes.data_as(ctypes.c_void_p),
                                    qv.ctypes.data_as(ctypes.c_void_p))
        ref = _vrr_reference(q, tuple(B))
        expect = np.array([ref(e, f, 0) for e in E.comps for f in F.comps])
        err = np.abs(acc - expect).max() / max(1.0, np.abs(expect).max())
        assert err < 1e-12, (name, err)


def test_generated_hrr_is_the_recurrence(gen, lib):
    rng = np.random.default_rng(11)
    for name, (la, lb, lc, ld) in _classes(gen):
        E, F = gen.Range(la, la + lb), gen.Range(lc, lc + ld)
        acc = rng.uniform(-1, 1, size=len(E) * len(F))
        AB, CD = rng.uniform(-2, 2, size=3), rng.uniform(-2, 2, size=3)
        A, Bc, C, D = gen.cart(la), gen.cart(lb), gen.cart(lc), gen.cart(ld)
        out = np.zeros(len(A) * len(Bc) * len(C) * len(D))
        getattr(lib, f"hrr_{name}")(acc.ctypes.data_as(ctypes.c_void_p), out.ctypes.data_as(ctypes.c_void_p),
                                    AB.ctypes.data_as(ctypes.c_void_p), CD.ctypes.data_as(ctypes.c_void_p))

        @lru_cache(maxsize=None)
        def val(a, b, c, d):
            if sum(d) > 0:
                i = next(k for k in range(3) if d[k] > 0)
                d1 = _lower(d, i)
                return val(a, b, _raise(c, i), d1) + CD[i] * val(a, b, c, d1)
            if sum(b) > 0:
                i = next(k for k in range(3) if b[k] > 0)
                b1 = _lower(b, i)
                return val(_raise(a, i), b1, c, d) + AB[i] * val(a, b1, c, d)
            return acc[E.index[a] * len(F) + F.index[c]]
        expect = np.array([val(a, b, c, d) for a in A for b in Bc for c in C for d in D])
        err = np.abs(out - expect).max() / max(1.0, np.abs(expect).max())
        assert err < 1e-12, (name, err)
