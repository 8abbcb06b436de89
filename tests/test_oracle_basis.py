"""Pins of the 1D rules (Section 2: GL nodal basis, (p+1)-point Gauss rule)."""
import numpy as np
import numpy.polynomial.legendre as npleg
import pytest

from oracle import basis


@pytest.mark.parametrize("n", range(1, 11))
def test_gauss_exact_to_degree_2n_minus_1(n):
    x, w = basis.gauss_legendre(n)
    assert abs(w.sum() - 1.0) < 1e-15
    for j in range(2 * n):
        assert abs(np.dot(w, x ** j) - 1.0 / (j + 1)) < 1e-14
    # and not exact one degree higher (it is an n-point rule)
    assert abs(np.dot(w, x ** (2 * n)) - 1.0 / (2 * n + 1)) > 1e-12


@pytest.mark.parametrize("n", range(1, 11))
def test_gauss_points_are_legendre_roots(n):
    x, _ = basis.gauss_legendre(n)
    c = np.zeros(n + 1)
    c[n] = 1.0
    assert np.max(np.abs(npleg.legval(2 * x - 1, c))) < 1e-13
    assert np.all(np.diff(x) > 0)


@pytest.mark.parametrize("n", range(2, 11))
def test_gauss_lobatto_nodes(n):
    x = basis.gauss_lobatto(n)
    assert x[0] == 0.0 and x[-1] == 1.0
    assert np.max(np.abs(x + x[::-1] - 1.0)) < 1e-15      # symmetric
    c = np.zeros(n)
    c[n - 1] = 1.0
    dP = npleg.legder(c)
    if n > 2:
        assert np.max(np.abs(npleg.legval(2 * x[1:-1] - 1, dP))) < 1e-12
    # the GL rule with these nodes is exact to degree 2n-3
    V = np.vander(x, n, increasing=True).T
    w = np.linalg.solve(V, 1.0 / np.arange(1, n + 1))
    for j in range(2 * n - 2):
        assert abs(np.dot(w, x ** j) - 1.0 / (j + 1)) < 1e-13


@pytest.mark.parametrize("n", range(2, 11))
def test_lagrange_cardinal_and_derivative_exact(n):
    nodes = basis.gauss_lobatto(n)
    L = basis.lagrange_values(nodes, nodes)
    assert np.max(np.abs(L - np.eye(n))) < 1e-13
    xs = np.linspace(0, 1, 17)
    D = basis.lagrange_derivatives(nodes, xs)
    assert np.max(np.abs(D.sum(axis=1))) < 1e-11        # annihilates constants
    for deg in range(n):                                 # exact up to degree n-1
        dv = D @ nodes ** deg
        exact = deg * xs ** (deg - 1) if deg > 0 else 0 * xs
        assert np.max(np.abs(dv - exact)) < 1e-10 * max(1, n ** 2)
