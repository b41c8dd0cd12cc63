"""The double-float ("df64") arithmetic of the CUDA path's df64 tier
(paper_1303_4916_gb300/csrc/df64.cuh), built for the host by
tests/df64_host_harness.cpp, against exact rational arithmetic.

A df64 value is hi + lo with two floats; the operations are the error-free
transformations (two-sum, FMA two-product) and must keep the unit roundoff
near 2^-48: the tier's claim of J/K within the FP64 tolerance rests on it.
Sums are bounded relative to the operands' magnitudes (the short double-float
addition), products and the fused multiply-add relative to their terms.
"""
import ctypes
import os
import random
import shutil
import subprocess
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1303_4916_gb300", "csrc")
U = Fraction(1, 2 ** 48)


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    cxx = shutil.which("g++")
    inc = "/usr/local/cuda/include"
    if not cxx or not os.path.isdir(inc):
        pytest.skip("no host C++ compiler or CUDA headers")
    out = str(tmp_path_factory.mktemp("df") / "libdf.so")
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-shared", "-fPIC", "-I", CSRC, "-I", inc,
                    os.path.join(ROOT, "tests", "df64_host_harness.cpp"), "-o", out], check=True)
    return ctypes.CDLL(out)


def _pair(x):
    """A normalised (hi, lo) float pair of the double x, and its exact value."""
    hi = np.float32(x)
    lo = np.float32(x - float(hi))
    return np.array([hi, lo], dtype=np.float32), Fraction(float(hi)) + Fraction(float(lo))


def _val(r):
    return Fraction(float(r[0])) + Fraction(float(r[1]))


def _call(fn, *args):
    r = np.zeros(2, dtype=np.float32)
    ptrs = [a.ctypes.data_as(ctypes.c_void_p) if isinstance(a, np.ndarray) else ctypes.c_float(a) for a in args]
    fn(*ptrs, r.ctypes.data_as(ctypes.c_void_p))
    return r


def _normalised(r):
    # |lo| <= ulp(hi) / 2
    return abs(float(r[1])) <= float(np.spacing(np.float32(abs(r[0])))) / 2


def _rel(x, exact):
    return abs(x - exact) / abs(exact)


def test_add_sub_mul_fma_within_a_few_units_of_2_to_minus_48(lib):
    rng = random.Random(3)
    worst = {"add": 0, "sub": 0, "mul": 0, "fma": 0, "mulf": 0}
    for _ in range(4000):
        e = rng.uniform(-20, 20)
        a, A = _pair(rng.uniform(0.5, 1.0) * 2.0 ** e * rng.choice((-1, 1)))
        b, B = _pair(rng.uniform(0.5, 1.0) * 2.0 ** rng.uniform(-20, 20) * rng.choice((-1, 1)))
        c, Cx = _pair(rng.uniform(-1, 1) * float(A * B) * 2.0 ** rng.uniform(-3, 3))
        f = np.float32(rng.uniform(-4, 4))
        for name, r, exact in (("add", _call(lib.df_add2, a, b), A + B),
                               ("sub", _call(lib.df_sub2, a, b), A - B),
                               ("mul", _call(lib.df_mul2, a, b), A * B),
                               ("fma", _call(lib.df_fma2, a, b, c), A * B + Cx),
                               ("mulf", _call(lib.df_mulf2, a, float(f)), A * Fraction(float(f)))):
            assert _normalised(r), (name, r)
            # the addition is the short ("sloppy") double-float sum: accurate
            # relative to the operands' magnitudes, not to a cancelled result
            scale = {"add": abs(A) + abs(B), "sub": abs(A) + abs(B), "mul": abs(A * B),
                     "mulf": abs(A * Fraction(float(f))), "fma": abs(A * B) + abs(Cx)}[name]
            if scale != 0:
                worst[name] = max(worst[name], abs(_val(r) - exact) / scale)
    for name, w in worst.items():
        assert w <= 4 * U, (name, float(w / U))


def test_conversion_and_rsqrt(lib):
    rng = random.Random(5)
    for _ in range(2000):
        x = rng.uniform(1e-3, 1e3)
        r = np.zeros(2, dtype=np.float32)
        lib.df_from_double(ctypes.c_double(x), r.ctypes.data_as(ctypes.c_void_p))
        assert _normalised(r) and _rel(_val(r), Fraction(x)) <= U   # 48 of x's 53 bits survive
        a, A = _pair(x)
        y = _call(lib.df_rsqrt2, a)
        # 1/sqrt(A) to within ~2^-45: check y^2 A against 1 exactly
        assert _rel(_val(y) ** 2 * A, Fraction(1)) <= 16 * U, x
