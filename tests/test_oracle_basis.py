"""Pins for oracle/basis.py: closed-form Gauss-Legendre rules, exactness."""
import numpy as np
import numpy.polynomial.polynomial as npoly
import pytest

from oracle.basis import Basis1D, gauss_legendre_01, lagrange_values


def test_gl_closed_forms():
    # textbook closed forms of the 1-, 2- and 3-point rules, mapped to [0, 1]
    x, w = gauss_legendre_01(1)
    assert np.allclose(x, [0.5]) and np.allclose(w, [1.0])
    x, w = gauss_legendre_01(2)
    assert np.allclose(x, [0.5 - np.sqrt(3) / 6, 0.5 + np.sqrt(3) / 6], atol=1e-15)
    assert np.allclose(w, [0.5, 0.5], atol=1e-15)
    x, w = gauss_legendre_01(3)
    assert np.allclose(x, [0.5 - np.sqrt(15) / 10, 0.5, 0.5 + np.sqrt(15) / 10], atol=1e-15)
    assert np.allclose(w, [5 / 18, 8 / 18, 5 / 18], atol=1e-15)


@pytest.mark.parametrize("n", [1, 2, 5, 8, 16, 31])
def test_gl_exact_degree(n):
    x, w = gauss_legendre_01(n)
    assert abs(w.sum() - 1.0) < 1e-14
    for k in range(2 * n):
        assert abs(np.dot(w, x ** k) - 1.0 / (k + 1)) < 1e-13
    # not exact at degree 2n: shows the test can fail
    assert abs(np.dot(w, x ** (2 * n)) - 1.0 / (2 * n + 1)) > 1e-8 * (0.25 ** n)


@pytest.mark.parametrize("n", [1, 2, 4, 8, 12])
def test_derivative_and_endpoints_exact(n):
    rng = np.random.default_rng(n)
    b = Basis1D(n)
    # collocated quadrature: G is the identity
    assert np.allclose(b.G, np.eye(n), atol=1e-13)
    for _ in range(3):
        c = rng.standard_normal(n)                 # degree n-1 polynomial
        vals = npoly.polyval(b.b, c)
        dvals = npoly.polyval(b.x, npoly.polyder(c))
        assert np.allclose(b.D @ vals, dvals, atol=1e-9 * max(1, np.abs(dvals).max()))
        assert abs(b.l0 @ vals - npoly.polyval(0.0, c)) < 1e-10
        assert abs(b.l1 @ vals - npoly.polyval(1.0, c)) < 1e-10
    assert np.allclose(b.D @ np.ones(n), 0.0, atol=1e-10 * n * n)


def test_overintegration_evaluation():
    b = Basis1D(4, mu=7)
    rng = np.random.default_rng(0)
    c = rng.standard_normal(4)
    assert np.allclose(b.G @ npoly.polyval(b.b, c), npoly.polyval(b.x, c), atol=1e-12)
    assert np.allclose(lagrange_values(b.b, b.b), np.eye(4), atol=1e-14)
