"""Pins of the oracle's 1D rules (Section 2.1: GLL interpolation nodes,
Gauss-Legendre quadrature, Lagrange basis) against closed forms and numpy."""
import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

import oracle
from meshutil import gll_nodes


def test_gll_closed_forms():
    np.testing.assert_allclose(oracle.gauss_lobatto(1), [-1, 1], atol=0)
    np.testing.assert_allclose(oracle.gauss_lobatto(2), [-1, 0, 1], atol=1e-15)
    s5 = 1 / np.sqrt(5)
    np.testing.assert_allclose(oracle.gauss_lobatto(3), [-1, -s5, s5, 1], atol=1e-15)
    s37 = np.sqrt(3 / 7)
    np.testing.assert_allclose(oracle.gauss_lobatto(4), [-1, -s37, 0, s37, 1], atol=1e-15)


@pytest.mark.parametrize("p", range(1, 15))
def test_gll_matches_numpy_roots(p):
    np.testing.assert_allclose(oracle.gauss_lobatto(p), gll_nodes(p), atol=2e-15)


def test_gauss_closed_form():
    x, w = oracle.gauss_legendre(3)
    np.testing.assert_allclose(x, [-np.sqrt(0.6), 0, np.sqrt(0.6)], atol=1e-15)
    np.testing.assert_allclose(w, [5 / 9, 8 / 9, 5 / 9], atol=1e-15)
    x, w = oracle.gauss_legendre(2)
    np.testing.assert_allclose(x, [-1 / np.sqrt(3), 1 / np.sqrt(3)], atol=1e-15)
    np.testing.assert_allclose(w, [1, 1], atol=1e-15)


@pytest.mark.parametrize("q", range(1, 17))
def test_gauss_matches_numpy_and_is_exact(q):
    x, w = oracle.gauss_legendre(q)
    xr, wr = npleg.leggauss(q)
    np.testing.assert_allclose(x, xr, atol=2e-15)
    np.testing.assert_allclose(w, wr, atol=2e-15)
    assert abs(w.sum() - 2.0) < 1e-14
    for k in range(2 * q):  # exact for degree <= 2q-1
        exact = 2.0 / (k + 1) if k % 2 == 0 else 0.0
        assert abs(np.dot(w, x ** k) - exact) < 1e-13


@pytest.mark.parametrize("p", range(1, 13))
def test_basis_1d_reproduces_polynomials(p):
    q = p + 2
    B, D = oracle.basis_1d(p, q)
    xn = oracle.gauss_lobatto(p)
    xg, _ = oracle.gauss_legendre(q)
    np.testing.assert_allclose(B.sum(axis=1), 1.0, atol=1e-13)
    np.testing.assert_allclose(D.sum(axis=1), 0.0, atol=1e-11)
    for k in range(p + 1):
        np.testing.assert_allclose(B @ xn ** k, xg ** k, atol=1e-13)
        dk = k * xg ** (k - 1) if k > 0 else np.zeros(q)
        np.testing.assert_allclose(D @ xn ** k, dk, atol=1e-11)


def test_lagrange_is_cardinal():
    xn = oracle.gauss_lobatto(6)
    for i, t in enumerate(xn):
        phi, _ = oracle.lagrange(xn, t)
        e = np.zeros(7)
        e[i] = 1
        np.testing.assert_allclose(phi, e, atol=1e-14)


@pytest.mark.parametrize("p", range(1, 13))
def test_every_lor_interval_holds_a_gauss_point(p):
    """Reading R1 needs every GLL sub-interval to contain >= 1 of the p+2
    Gauss points, and no Gauss point may sit on a GLL node (no tie)."""
    xn = oracle.gauss_lobatto(p)
    xg, _ = oracle.gauss_legendre(p + 2)
    bins = np.searchsorted(xn[1:-1], xg, side="left")
    assert set(bins.tolist()) == set(range(p))
    assert np.min(np.abs(xg[:, None] - xn[None, 1:-1])) > 1e-3 if p > 1 else True
