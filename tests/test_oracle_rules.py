"""Pins for the oracle's 1D rules: Gauss-Legendre, Gauss-Lobatto, Lagrange basis."""
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("q", range(1, 10))
def test_gauss_exactness(orc, q):
    x, w = orc.gauss(q)
    assert abs(w.sum() - 1.0) < 1e-14
    for k in range(2 * q):
        assert abs((w * x ** k).sum() - 1.0 / (k + 1)) < 1e-14
    # a q-point rule is not exact for degree 2q (guards against a rule with more points)
    assert abs((w * x ** (2 * q)).sum() - 1.0 / (2 * q + 1)) > 1e-13


@pytest.mark.parametrize("q", range(1, 10))
def test_gauss_matches_numpy(orc, q):
    t, wt = np.polynomial.legendre.leggauss(q)
    x, w = orc.gauss(q)
    assert np.allclose(x, 0.5 * (1 + t), atol=1e-14)
    assert np.allclose(w, 0.5 * wt, atol=1e-14)


def test_gll_closed_forms(orc):
    for line in open(os.path.join(GOLDEN, "gll_nodes.txt")):
        if line.startswith("#") or not line.strip():
            continue
        vals = [float(v) for v in line.split()]
        p, t = int(vals[0]), np.array(vals[1:])
        assert np.allclose(orc.gll(p), 0.5 * (1 + t), atol=1e-15)


@pytest.mark.parametrize("p", range(1, 9))
def test_gll_are_roots_of_legendre_derivative(orc, p):
    cp = np.zeros(p + 1)
    cp[p] = 1.0
    roots = np.sort(np.polynomial.legendre.Legendre(cp).deriv().roots().real)
    x = orc.gll(p)
    assert x[0] == 0.0 and x[-1] == 1.0
    assert np.allclose(x[1:-1], 0.5 * (1 + roots), atol=1e-13)


@pytest.mark.parametrize("p", range(1, 9))
def test_lagrange_basis(orc, p):
    nodes = orc.gll(p)
    n = p + 1
    for j, xj in enumerate(nodes):
        l, _ = orc.lagrange(nodes, xj)
        assert np.allclose(l, np.eye(n)[j], atol=1e-13)
    for xi in np.linspace(0, 1, 7):
        l, dl = orc.lagrange(nodes, xi)
        assert abs(l.sum() - 1) < 1e-12 and abs(dl.sum()) < 1e-10
        # the basis reproduces monomials and their derivatives up to degree p
        for k in range(p + 1):
            assert abs((l * nodes ** k).sum() - xi ** k) < 1e-12
            dk = k * xi ** (k - 1) if k > 0 else 0.0
            assert abs((dl * nodes ** k).sum() - dk) < 1e-10
