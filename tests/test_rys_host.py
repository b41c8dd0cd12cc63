"""The Rys quadrature rule behind the f/g classes (host code of the library,
no GPU) against what the mathematics fixes: the rule is the Gauss rule of
the weight exp(-T t^2) on t in [0, 1] in u = t^2, so its moments are Boys
functions (checked against the oracle's Boys), it integrates polynomials of
degree 2n - 1 exactly (checked against a brute-force Gauss-Legendre
quadrature of the defining integral), and its one-point form is
u = F_1 / F_0, w = F_0."""
import numpy as np
import pytest

import oracle

TS = [0.0, 1e-3, 0.37, 2.5, 7.77, 19.9, 33.3, 45.1, 59.999, 60.0, 75.0, 300.0, 1e4]


@pytest.fixture(scope="module")
def rule():
    from paper_1303_4916_gb300 import build
    build.build()
    from paper_1303_4916_gb300 import hf_rys_rule
    return hf_rys_rule


@pytest.mark.parametrize("n", range(1, 10))
def test_moments_are_boys_functions(rule, n):
    for T in TS:
        u, w = rule(n, T)
        # below T = 60 the tabulated rule is exact to degree 2n - 1; above it
        # the Gauss-Hermite limit is exact for the degrees < n that an ERI
        # of n roots needs (the integral beyond t = 1 is below 1e-16 there)
        kmax = 2 * n if T < 60.0 else n
        for k in range(kmax):
            ref = oracle.boys(k, T)
            got = float(np.sum(w * u ** k))
            assert abs(got - ref) <= 1e-14 * ref, (n, T, k, got, ref)


def test_rule_integrates_polynomials_like_brute_force_quadrature(rule):
    x, gw = np.polynomial.legendre.leggauss(80)   # accurate to ~5e-16 here for these T
    t = 0.5 * (x + 1.0)
    rng = np.random.default_rng(3)
    for n in (1, 2, 4, 7, 9):
        for T in (0.05, 3.3, 12.0, 41.0):
            c = rng.normal(size=2 * n)          # f(u) = sum_k c_k u^k, degree 2n - 1
            ref = float(np.sum(0.5 * gw * np.polyval(c[::-1], t * t) * np.exp(-T * t * t)))
            u, w = rule(n, T)
            got = float(np.sum(w * np.polyval(c[::-1], u)))
            scale = float(np.sum(0.5 * gw * np.abs(np.polyval(np.abs(c[::-1]), t * t)) * np.exp(-T * t * t)))
            assert abs(got - ref) <= 1e-14 * scale, (n, T)


def test_one_point_rule_closed_form(rule):
    for T in (0.0, 0.8, 9.0, 59.0, 61.0, 500.0):
        u, w = rule(1, T)
        F0, F1 = oracle.boys(0, T), oracle.boys(1, T)
        assert w[0] == pytest.approx(F0, rel=1e-14)
        if T < 60.0:
            assert u[0] == pytest.approx(F1 / F0, rel=1e-14)
        else:  # Hermite limit: u = 1/(2T), w = sqrt(pi)/2 / sqrt(T)
            assert u[0] == pytest.approx(0.5 / T, rel=1e-14)


def test_roots_ascending_inside_the_interval_and_weights_positive(rule):
    for n in range(1, 10):
        for T in TS:
            u, w = rule(n, T)
            assert np.all(u > 0) and np.all(u < 1) and np.all(np.diff(u) > 0), (n, T)
            assert np.all(w > 0)


def test_invalid_arguments(rule):
    from paper_1303_4916_gb300 import HFError
    for n, T in ((0, 1.0), (10, 1.0), (3, -1.0), (3, float("nan")), (3, float("inf"))):
        with pytest.raises(HFError) as e:
            rule(n, T)
        assert e.value.code == -1
