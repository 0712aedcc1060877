"""Pins for theta_m(tol) (oracle/theta_tables.json, oracle/make_theta.py).

* SciPy ships the published double-precision theta_m of Al-Mohy & Higham
  (their Table 3.1 and Higham's Table A.3, 2-3 significant digits); the
  oracle's values, computed from the backward-error definition, must round to
  them.
* m = 1 has a closed form: h_2(x) = log(1 + x) - x, so
  htilde_2(x)/x = (-log(1 - x) - x)/x, whose root at tol is found independently.
* The Taylor coefficients of log(exp(-x) T_m(x)) are checked against sympy.
"""
import math

import numpy as np
import pytest
from scipy.optimize import brentq

from oracle import expmv


def test_theta_double_matches_published_table():
    mod = pytest.importorskip("scipy.sparse.linalg._expm_multiply")
    published = mod._theta
    for m, ref in published.items():
        if m == 1:
            continue  # the printed 2.29e-16 is not the root of the definition; see closed form below
        got = expmv.THETA["double"][m]
        digits = 2 if m >= 35 else 3
        scale = 10 ** (math.floor(math.log10(ref)) - digits + 1)
        # within one unit of the last printed digit (m = 8 prints 5.00e-2 for
        # a root at 4.991e-2; every other entry also rounds correctly)
        assert abs(got - ref) <= scale, (m, got, ref)


@pytest.mark.parametrize("precision", ["double", "single"])
def test_theta_1_closed_form(precision):
    tol = expmv.TOL[precision]
    # (-log(1-x) - x)/x = x/2 + x^2/3 + x^3/4 + ...; summed term by term to
    # avoid the cancellation of the closed form at x ~ 1e-16.
    f = lambda x: sum(x ** (k - 1) / k for k in range(2, 40)) - tol
    root = brentq(f, tol, 4 * tol, xtol=1e-30, rtol=1e-14)
    assert abs(expmv.THETA[precision][1] - root) <= 1e-12 * root


def test_theta_monotone_and_single_larger():
    for prec in ("double", "single"):
        th = [expmv.THETA[prec][m] for m in range(1, 56)]
        assert all(b > a for a, b in zip(th, th[1:]))
    assert all(expmv.THETA["single"][m] > expmv.THETA["double"][m] for m in range(1, 56))


def test_log_series_coefficients_against_sympy():
    sympy = pytest.importorskip("sympy")
    mpmath = pytest.importorskip("mpmath")
    from oracle import make_theta
    x = sympy.symbols("x")
    for m in (2, 3, 5):
        Tm = sum(x ** j / sympy.factorial(j) for j in range(m + 1))
        ser = sympy.series(sympy.log(sympy.exp(-x) * Tm), x, 0, 3 * m + 4).removeO()
        coeffs = make_theta.log_series(m, 3 * m + 3)
        for k in range(1, 3 * m + 4):
            ref = sympy.Rational(ser.coeff(x, k))
            assert abs(float(coeffs[k]) - float(ref)) <= 1e-25 + 1e-20 * abs(float(ref)), (m, k)
