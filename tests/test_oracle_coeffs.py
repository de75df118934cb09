"""Pins for the oracle's Chebyshev coefficients (Sec. 2.1) and the bounds of Sec. 4.

The coefficients are checked against an independent derivation: the Chebyshev
series of log on [a, b] in closed form, aliased onto degree n the way the n+1
first-kind nodes alias T_m (T_{2l(n+1) +- j} = (-1)^l T_j and T_{n+1} = 0 on the
nodes).  With alpha = (a+b)/(b-a) and r = alpha - sqrt(alpha^2 - 1):
    log(((b-a) y + a + b)/2) = log((b-a)/2) - log(2r) + sum_k 2 (-1)^{k+1} r^k T_k(y) / k.
"""
import json
import os

import numpy as np
import numpy.polynomial.chebyshev as npc
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def series_log(a, b, kmax):
    alpha = (a + b) / (b - a)
    r = alpha - np.sqrt(alpha * alpha - 1.0)
    s = np.zeros(kmax + 1)
    s[0] = np.log((b - a) / 2.0) - np.log(2.0 * r)
    k = np.arange(1, kmax + 1)
    s[1:] = 2.0 * (-1.0) ** (k + 1) * r ** k / k
    return s


def aliased(a, b, n):
    N = n + 1
    kmax = 400 * N
    s = series_log(a, b, kmax)
    c = np.zeros(n + 1)
    for j in range(n + 1):
        acc = s[j]
        l = 1
        while 2 * l * N + j <= kmax:
            sign = (-1.0) ** l
            if j == 0:
                acc += sign * s[2 * l * N]
            else:
                acc += sign * (s[2 * l * N - j] + s[2 * l * N + j])
            l += 1
        c[j] = acc
    return c


@pytest.mark.parametrize("n,a,b", [(0, 0.1, 0.9), (1, 0.1, 0.9), (2, 0.3, 2.0), (10, 0.1, 0.9),
                                   (30, 0.0325, 0.99), (50, 0.1, 8.1), (100, 0.01, 0.99)])
def test_coeffs_match_aliased_closed_form(oracle_mod, n, a, b):
    c = oracle_mod.cheb_coeffs(n, a, b)
    ref = aliased(a, b, n)
    scale = max(1.0, np.max(np.abs(ref)))
    np.testing.assert_allclose(c, ref, rtol=0, atol=2e-13 * scale * (n + 1))


@pytest.mark.parametrize("n", [0, 1, 5, 17])
def test_interpolates_at_nodes(oracle_mod, n):
    a, b = 0.05, 3.0
    c = oracle_mod.cheb_coeffs(n, a, b)
    xk = np.cos(np.pi * (np.arange(n + 1) + 0.5) / (n + 1))
    np.testing.assert_allclose(npc.chebval(xk, c), np.log(((b - a) * xk + a + b) / 2), rtol=0, atol=1e-13)


@pytest.mark.parametrize("delta,n", [(0.1, 5), (0.1, 14), (0.05, 20), (0.2, 8), (0.01, 60)])
def test_chebyshev_error_bound(oracle_mod, delta, n):
    """Sec. 4.1: |log(1-x) - p_n(x)| <= 20 log(2(1/delta-1)) / ((K-1) K^n) on [delta, 1-delta]."""
    c = oracle_mod.cheb_coeffs(n, delta, 1.0 - delta)  # log on [delta, 1-delta]; x -> 1-x symmetric
    y = np.linspace(delta, 1.0 - delta, 20001)
    ymap = (2.0 * y - 1.0) / (1.0 - 2.0 * delta)
    err = np.max(np.abs(npc.chebval(ymap, c) - np.log(y)))
    assert err <= oracle_mod.chebyshev_error_bound(delta, n)


def test_lemma2_negative_polynomial(oracle_mod):
    """Lemma 2: p_n < 0 on [delta, 1-delta] once the bound is below log(1/(1-delta))."""
    delta = 0.1
    n = next(k for k in range(1, 200) if oracle_mod.chebyshev_error_bound(delta, k) <= np.log(1 / (1 - delta)))
    c = oracle_mod.cheb_coeffs(n, delta, 1.0 - delta)
    y = np.linspace(delta, 1.0 - delta, 20001)
    assert np.all(npc.chebval((2 * y - 1) / (1 - 2 * delta), c) < 0)


def test_alg1_coefficients_are_reflection(oracle_mod):
    """Algorithm 1's function log(1 - ((1-2 delta)x+1)/2) is the [delta,1-delta]
    logarithm at -x, and the nodes are symmetric, so c^alg1_j = (-1)^j c_j."""
    for delta, n in [(0.1, 14), (0.3, 7), (0.02, 40)]:
        c = oracle_mod.cheb_coeffs(n, delta, 1 - delta)
        c1 = oracle_mod.cheb_coeffs_alg1(n, delta)
        np.testing.assert_allclose(c1, (-1.0) ** np.arange(n + 1) * c, rtol=0, atol=1e-13)


def test_theorem1_worked_example(oracle_mod):
    """Theorem 1's degree condition at the paper's worked example (delta=0.1, eps=0.01).

    The right-hand side of the condition is exactly the n at which the Sec. 4
    inequality (eq1) 20 log(2(1/delta-1)) / ((K-1)K^n) <= (eps/2) log(1/(1-delta))
    starts to hold, so the smallest integer n meeting one meets the other.  The
    paper's text prints n = 14 for this example; the formula gives 26 (see the
    fixture for the reading)."""
    g = json.load(open(os.path.join(GOLDEN, "thm1_worked_example.json")))
    delta, eps = g["delta"], g["eps"]
    rhs = oracle_mod.thm1_degree(delta, eps)
    n_formula = int(np.ceil(rhs))
    lhs = lambda n: oracle_mod.chebyshev_error_bound(delta, n)
    target = eps / 2 * np.log(1 / (1 - delta))
    n_eq1 = next(k for k in range(1, 500) if lhs(k) <= target)
    assert n_formula == n_eq1 == g["formula_n"]
    assert g["paper_printed_n"] == 14 and g["paper_printed_n"] != n_formula
