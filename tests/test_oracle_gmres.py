"""Pins for oracle/gmres.py."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import synthetic
from oracle.dg import AdvectionDG, PeriodicMesh
from oracle.gmres import gmres
from oracle.precond import block_jacobi, kron_dense


def test_exact_inverse_converges_in_one_iteration():
    rng = np.random.default_rng(0)
    blocks = [rng.standard_normal((5, 5)) + 5 * np.eye(5) for _ in range(6)]
    A = sp.block_diag(blocks).tocsr()
    inv = np.linalg.inv(A.toarray())
    b = rng.standard_normal(30)
    x, info = gmres(lambda v: A @ v, b, M=lambda v: inv @ v, rtol=1e-12)
    assert info["iters"] == 1 and info["converged"]
    assert np.allclose(A @ x, b, atol=1e-11)


def test_matches_sparse_direct_solve():
    dg = AdvectionDG(PeriodicMesh((4, 4)), 4, 0.1, synthetic.fourier_velocity(3, 2))
    S = dg.global_matrix()
    b = synthetic.rhs(1, dg.ndof)
    xs = spla.spsolve(S.tocsc(), b)
    for rtol, tol in [(1e-8, 1e-6), (1e-12, 1e-9)]:
        x, info = gmres(lambda v: S @ v, b, M=block_jacobi(dg), rtol=rtol)
        assert info["converged"] and info["true_rel_res"] <= rtol
        assert np.linalg.norm(x - xs) <= tol * np.linalg.norm(xs)
        xf, infof = gmres(lambda v: S @ v, b, M=block_jacobi(dg), rtol=rtol, flexible=True)
        assert infof["iters"] == info["iters"]
        assert np.linalg.norm(xf - xs) <= tol * np.linalg.norm(xs)


def test_restart_and_unpreconditioned():
    dg = AdvectionDG(PeriodicMesh((3, 3)), 3, 0.05, synthetic.fourier_velocity(6, 2))
    S = dg.global_matrix()
    b = synthetic.rhs(2, dg.ndof)
    x, info = gmres(lambda v: S @ v, b, restart=5, rtol=1e-10, max_iters=5000)
    assert info["converged"] and info["iters"] > 5
    assert np.linalg.norm(S @ x - b) <= 1e-10 * np.linalg.norm(b)


def test_jacobi_and_kronecker_iterations_identical_for_constant_velocity():
    # Sec. 5.1: when the blocks are exact Kronecker sums the two preconditioners
    # coincide and so do the GMRES iteration counts
    dg = AdvectionDG(PeriodicMesh((4, 4)), 5, 0.1, synthetic.constant_velocity([1.0, 0.5]))
    S = dg.global_matrix()
    b = synthetic.rhs(1704, dg.ndof)
    _, iJ = gmres(lambda v: S @ v, b, M=block_jacobi(dg), rtol=1e-8)
    _, iK = gmres(lambda v: S @ v, b, M=kron_dense(dg), rtol=1e-8)
    assert iJ["converged"] and iK["converged"] and iJ["iters"] == iK["iters"]


def test_zero_rhs():
    x, info = gmres(lambda v: 2 * v, np.zeros(4))
    assert info["converged"] and info["iters"] == 0 and not x.any()


@pytest.mark.parametrize("p", [1, 3, 6])
@pytest.mark.parametrize("field", ["constant", "separable"])
def test_jacobi_and_kronecker_identical_on_cartesian_grid_table(p, field):
    """Table adv-results (Cartesian grid, velocity fields (a) constant and (b)
    separable, dt = 0.5, p = 1..10): J and K take identical GMRES iteration counts,
    because every diagonal block is an exact two-term Kronecker sum (Eqs.
    adv-kron-const, adv-kron-cart).  The paper's mesh is shown only as a figure, so
    the counts themselves are not compared; the identity is."""
    vel = (synthetic.constant_velocity([1.0, 2.0]) if field == "constant"
           else synthetic.fourier_velocity(31, 2, separable=True))
    dg = AdvectionDG(PeriodicMesh((4, 4)), p + 1, 0.5, vel)
    S = dg.global_matrix()
    b = synthetic.rhs(1704, dg.ndof)
    _, iJ = gmres(lambda v: S @ v, b, M=block_jacobi(dg), rtol=1e-8)
    _, iK = gmres(lambda v: S @ v, b, M=kron_dense(dg), rtol=1e-8)
    assert iJ["converged"] and iK["converged"] and iJ["iters"] == iK["iters"], (iJ, iK)
