"""Pins of the oracle's reference tables against definitions independent of it.

- Dubiner basis (Sec. 2.2, Eq. dubiner) against scipy's Jacobi polynomials.
- Mass-matrix orthogonality and norms against exact sympy integration.
- Quadrature rules against exact monomial integrals over the reference triangle
  and numpy's Gauss-Legendre nodes.
"""
import itertools

import numpy as np
import pytest
import sympy as sp
from scipy.special import eval_jacobi, eval_legendre

import oracle

MODES = [(0, 0), (1, 0), (0, 1), (2, 0), (1, 1), (0, 2)]


def dubiner_scipy(i, j, xi, eta):
    a = 2.0 * (1.0 + xi) / (1.0 - eta) - 1.0
    b = eta
    return eval_legendre(i, a) * ((1.0 - b) / 2.0) ** i * eval_jacobi(j, 2 * i + 1, 0, b)


def test_basis_matches_jacobi_definition():
    rng = np.random.default_rng(0)
    for _ in range(200):
        u, v = rng.random(2)
        if u + v > 1:
            u, v = 1 - u, 1 - v
        xi, eta = -1 + 2 * u, -1 + 2 * v
        phi, dxi, deta = oracle.basis(2, xi, eta)
        h = 1e-6
        fp, _, _ = oracle.basis(2, xi + h, eta)
        fm, _, _ = oracle.basis(2, xi - h, eta)
        gp, _, _ = oracle.basis(2, xi, eta + h)
        gm, _, _ = oracle.basis(2, xi, eta - h)
        for k, (i, j) in enumerate(MODES):
            assert phi[k] == pytest.approx(dubiner_scipy(i, j, xi, eta), abs=1e-12)
            assert dxi[k] == pytest.approx((fp[k] - fm[k]) / (2 * h), abs=1e-8)
            assert deta[k] == pytest.approx((gp[k] - gm[k]) / (2 * h), abs=1e-8)


def _exact_mass_matrix():
    x, y = sp.symbols("x y")
    a = 2 * (1 + x) / (1 - y) - 1
    polys = []
    for i, j in MODES:
        e = sp.legendre(i, a) * ((1 - y) / 2) ** i * sp.jacobi(j, 2 * i + 1, 0, y)
        polys.append(sp.expand(sp.cancel(sp.simplify(e))))
    M = sp.zeros(6, 6)
    for p, q in itertools.product(range(6), range(6)):
        M[p, q] = sp.integrate(sp.integrate(polys[p] * polys[q], (x, -1, -y)), (y, -1, 1))
    return M


def test_mass_matrix_diagonal_with_stated_norms():
    M = _exact_mass_matrix()
    norms = [sp.Rational(2), sp.Rational(1, 3), sp.Rational(1), sp.Rational(2, 15), sp.Rational(2, 9),
             sp.Rational(2, 3)]
    for p in range(6):
        for q in range(6):
            assert M[p, q] == (norms[p] if p == q else 0)
    # the oracle's p=2 area rule integrates the basis products (degree 4) exactly
    xi, eta, w = oracle.area_rule(2)
    vals = np.array([oracle.basis(2, a, b)[0] for a, b in zip(xi, eta)])
    Mq = (vals * w[:, None]).T @ vals
    assert np.allclose(Mq, np.array(M.tolist(), dtype=float), atol=1e-14)


def _exact_monomial(a, b):
    x, y = sp.symbols("x y")
    return float(sp.integrate(sp.integrate(x ** a * y ** b, (x, -1, -y)), (y, -1, 1)))


@pytest.mark.parametrize("p,degree", [(1, 4), (2, 6)])
def test_area_rule_exact_to_degree(p, degree):
    xi, eta, w = oracle.area_rule(p)
    assert len(w) == (6 if p == 1 else 12)
    assert np.all(w > 0)
    # interior points
    assert np.all(xi > -1) and np.all(eta > -1) and np.all(xi + eta < 0)
    for a in range(degree + 1):
        for b in range(degree + 1 - a):
            got = np.sum(w * xi ** a * eta ** b)
            assert got == pytest.approx(_exact_monomial(a, b), abs=2e-14), (a, b)
    # and not exact one degree higher (the rule is the one stated, not a stronger one)
    errs = [abs(np.sum(w * xi ** a * eta ** (degree + 1 - a)) - _exact_monomial(a, degree + 1 - a))
            for a in range(degree + 2)]
    assert max(errs) > 1e-8


def test_high_order_rule_exact_to_degree_14():
    xi, eta, w = oracle.high_rule()
    for a in range(15):
        for b in range(15 - a):
            assert np.sum(w * xi ** a * eta ** b) == pytest.approx(_exact_monomial(a, b), abs=1e-13)


@pytest.mark.parametrize("n", [2, 4])
def test_edge_rule_is_gauss_legendre(n):
    s, w = oracle.edge_rule(n)
    xr, wr = np.polynomial.legendre.leggauss(n)
    assert np.allclose(s, xr, atol=1e-15, rtol=0)
    assert np.allclose(w, wr, atol=1e-15, rtol=0)
    assert np.all(s[::-1] == -s)  # mirror symmetric, used to match the two sides of an edge
