"""Pins for the oracle's quadrature rules: exactness on monomials (closed form)
and agreement of Golub-Welsch with numpy's Gauss-Legendre routine."""
from math import factorial

import numpy as np
import pytest

from oracle.quadrature import gauss_legendre, near_rule, rule_degree, triangle_rule


def exact_monomial(a, b):
    # area-normalised integral of lambda_2^a lambda_3^b over a triangle
    return 2.0 * factorial(a) * factorial(b) / factorial(a + b + 2)


def integrate(bary, w, a, b):
    return float(np.sum(w * bary[:, 1] ** a * bary[:, 2] ** b))


@pytest.mark.parametrize("k", [1, 3, 4, 7, 20])
def test_rule_exact_to_degree(k):
    bary, w = near_rule() if k == 20 else triangle_rule(k)
    assert len(w) == k
    assert np.allclose(bary.sum(1), 1.0)
    assert abs(w.sum() - 1.0) < 1e-14
    deg = rule_degree(k)
    for tot in range(deg + 1):
        for a in range(tot + 1):
            assert abs(integrate(bary, w, a, tot - a) - exact_monomial(a, tot - a)) < 1e-14


@pytest.mark.parametrize("k", [1, 3, 4, 7])
def test_rule_not_exact_beyond_degree(k):
    bary, w = triangle_rule(k)
    deg = rule_degree(k) + 1
    errs = [abs(integrate(bary, w, a, deg - a) - exact_monomial(a, deg - a)) for a in range(deg + 1)]
    assert max(errs) > 1e-6


@pytest.mark.parametrize("n", [1, 2, 4, 5, 9, 16])
def test_gauss_legendre_matches_numpy(n):
    x, w = gauss_legendre(n)
    xr, wr = np.polynomial.legendre.leggauss(n)
    assert np.allclose(np.sort(x), 0.5 * (xr + 1.0), atol=1e-14)
    assert np.allclose(w[np.argsort(x)], 0.5 * wr, atol=1e-14)


@pytest.mark.parametrize("nu", [3, 4, 5, 6, 7])
def test_collapsed_near_rules(nu):
    # the near rules of nu x (nu - 1) points (the near_k option; 5 x 4 = 20 by default) integrate
    # every monomial to total degree 2 nu - 3 and miss one degree above
    bary, w = near_rule(nu, nu - 1)
    k = nu * (nu - 1)
    assert len(w) == k and abs(w.sum() - 1.0) < 1e-14
    deg = rule_degree(k)
    assert deg == 2 * nu - 3
    for tot in range(deg + 1):
        for a in range(tot + 1):
            assert abs(integrate(bary, w, a, tot - a) - exact_monomial(a, tot - a)) < 1e-14
    errs = [abs(integrate(bary, w, a, deg + 1 - a) - exact_monomial(a, deg + 1 - a)) for a in range(deg + 2)]
    assert max(errs) > 1e-9
