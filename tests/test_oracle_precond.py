"""Pins for oracle/precond.py: Schur/Sylvester routes agree with dense LU."""
import numpy as np
import pytest

import synthetic
from oracle.dg import AdvectionDG, PeriodicMesh
from oracle.ksvd import ksvd_2d, ksvd_3d_nested, kron_sum
from oracle.precond import apply_2d, apply_3d, apply_dense, factor_2d, factor_3d


@pytest.mark.parametrize("n", [1, 2, 3, 7])
def test_2d_paper_route_random_factors(n):
    rng = np.random.default_rng(n)
    A1, B1, A2, B2 = (rng.standard_normal((n, n)) + 3 * np.eye(n) for _ in range(4))
    P = np.kron(A1, B1) + np.kron(A2, B2)
    b = rng.standard_normal(n * n)
    x = apply_2d(factor_2d(A1, B1, A2, B2), b)
    assert np.allclose(P @ x, b, atol=1e-11 * np.abs(b).max())
    assert np.allclose(x, np.linalg.inv(P) @ b, rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("n", [4, 8, 16])
def test_2d_paper_route_advection(n):
    dg = AdvectionDG(PeriodicMesh((4, 4)), n, 0.05, synthetic.fourier_velocity(1705, 2))
    S = dg.element_block(5)
    _, As, Bs = ksvd_2d(S, n)
    P = kron_sum(As, Bs)
    b = np.random.default_rng(0).standard_normal(n * n)
    x1 = apply_dense(P, b)
    x2 = apply_2d(factor_2d(As[0], Bs[0], As[1], Bs[1]), b)
    assert np.linalg.norm(x1 - x2) <= 1e-12 * np.linalg.norm(x1) * max(1.0, np.linalg.cond(P) / 1e3)


@pytest.mark.parametrize("n", [2, 3, 5])
def test_3d_paper_route(n):
    rng = np.random.default_rng(n)
    A1, B1, C1, B2, C2 = (rng.standard_normal((n, n)) + 3 * np.eye(n) for _ in range(5))
    P = np.kron(A1, np.kron(B1, C1) + np.kron(B2, C2))
    b = rng.standard_normal(n ** 3)
    x = apply_3d(factor_3d(A1, B1, C1, B2, C2), b)
    assert np.allclose(P @ x, b, atol=1e-10 * np.abs(b).max())


def test_3d_paper_route_advection():
    n = 4
    dg = AdvectionDG(PeriodicMesh((2, 2, 2)), n, 0.05, synthetic.fourier_velocity(1707, 3))
    out = ksvd_3d_nested(dg.element_block(3), n)
    b = np.random.default_rng(1).standard_normal(n ** 3)
    x1 = apply_dense(out["P"], b)
    x2 = apply_3d(factor_3d(out["A1"], out["B1"], out["C1"], out["B2"], out["C2"]), b)
    assert np.linalg.norm(x1 - x2) <= 1e-11 * np.linalg.norm(x1)


def test_zero_dt_reduces_to_mass():
    n = 5
    dg = AdvectionDG(PeriodicMesh((2, 2)), n, 0.0, synthetic.fourier_velocity(2, 2))
    S = dg.element_block(0)
    s, As, Bs = ksvd_2d(S, n)
    assert s[1] / s[0] < 1e-15          # mass h^2 W (x) W is a single Kronecker product
    assert np.allclose(kron_sum(As, Bs), S, atol=1e-15)
