"""Pins of the time-integration oracle: Alexander's DIRK coefficients against the
order conditions and L-stability, observed orders of accuracy against the exact
semi-discrete solution, and conservation."""
import numpy as np
import pytest

import synthetic
from oracle import timestep as T
from oracle.dg import AdvectionDG, PeriodicMesh


def test_dirk3_coefficients():
    A, b, c = T.alexander_dirk3()
    g = A[0, 0]
    assert abs(g - 0.435866521508459) <= 1e-14        # Alexander's gamma
    assert np.allclose(A.sum(axis=1), c, rtol=0, atol=1e-15)
    one = np.ones(3)
    assert abs(b @ one - 1.0) <= 1e-15
    assert abs(b @ c - 0.5) <= 1e-15
    assert abs(b @ c ** 2 - 1.0 / 3.0) <= 1e-15
    assert abs(b @ A @ c - 1.0 / 6.0) <= 1e-15
    # a fourth-order condition fails (it is a third-order method)
    assert abs(b @ c ** 3 - 0.25) > 1e-3
    # stability function R(z) = 1 + z b^T (I - z A)^-1 1 vanishes at infinity
    for z in (-1e6, -1e9):
        R = 1.0 + z * b @ np.linalg.solve(np.eye(3) - z * A, one)
        assert abs(R) <= 10.0 / abs(z)
    # and |R| <= 1 on the imaginary axis (A-stability sample)
    for y in (0.1, 1.0, 10.0, 100.0):
        z = 1j * y
        R = 1.0 + z * b @ np.linalg.solve(np.eye(3) - z * A, one)
        assert abs(R) <= 1.0 + 1e-12


@pytest.fixture(scope="module")
def problem():
    dg = AdvectionDG(PeriodicMesh((3, 3), 1.0), 4, 0.05, synthetic.fourier_velocity(1705, 2, kmax=1))
    m, J = T.spatial_operator(dg)
    u0 = synthetic.rhs(1715, dg.ndof)
    return m, J, u0


@pytest.mark.parametrize("method,order,dt", [(T.backward_euler, 1, 0.02), (T.dirk3, 3, 0.05),
                                             (T.rk4, 4, 0.005)])
def test_observed_order(problem, method, order, dt):
    m, J, u0 = problem
    t_end = 0.2
    ref = T.exact(m, J, u0, t_end)
    errs = []
    for k in (1, 2):
        h = dt / k
        errs.append(np.linalg.norm(method(m, J, u0, h, int(round(t_end / h))) - ref))
    rate = np.log2(errs[0] / errs[1])
    assert abs(rate - order) <= 0.3, (errs, rate)


@pytest.mark.parametrize("method,dt", [(T.backward_euler, 0.05), (T.dirk3, 0.05), (T.rk4, 0.002)])
def test_conservation(problem, method, dt):
    """1^T J = 0 on a periodic mesh, so every method keeps 1^T M u."""
    m, J, u0 = problem
    u = method(m, J, u0, dt, 10)
    assert abs(m @ u - m @ u0) <= 1e-12 * np.abs(m * u0).sum()


def test_spatial_operator_matches_definition(problem):
    """S = M - dt J recovered: J from the assembled S, M the collocated mass."""
    dg = AdvectionDG(PeriodicMesh((3, 3), 1.0), 4, 0.05, synthetic.fourier_velocity(1705, 2, kmax=1))
    m, J = T.spatial_operator(dg)
    S = dg.global_matrix()
    x = synthetic.rhs(3, dg.ndof)
    assert np.linalg.norm(m * x - 0.05 * (J @ x) - S @ x) <= 1e-13 * np.linalg.norm(S @ x)
    # constant velocity: J 1 = 0 (free stream preserved)
    dgc = AdvectionDG(PeriodicMesh((3, 3), 1.0), 4, 0.05, synthetic.constant_velocity([1.0, 0.5]))
    _, Jc = T.spatial_operator(dgc)
    assert np.abs(Jc @ np.ones(dgc.ndof)).max() <= 1e-12
