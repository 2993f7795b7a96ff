"""GPU parity: curved (non-affine) 2D elements through tpp_set_metric_terms against the
oracle's mapped-element assembly (oracle/curved.py): the operator (collocated and
over-integrated, FP64 and FP32), the KSVD factors of the curved blocks and their apply,
exact block Jacobi, and GMRES."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla
import torch

import synthetic
from oracle.curved import CurvedAdvectionDG
from oracle.dg import AdvectionDG, PeriodicMesh
from oracle.gmres import gmres
from oracle.precond import kron_dense
from paper_1704_04549_gb300 import (TPP_FEAT_BLOCK_JACOBI, TPP_FEAT_MIXED, TPP_FEAT_TWO_SIDED,
                                    TPP_PC_KRON, mesh)
from tests.gpu_util import DEV, FP64_TOL, rel, to_dev, to_host
from tests.test_gpu_factors import _check_elements

pytestmark = pytest.mark.gpu

L = 2.0


def _warp(X):
    return synthetic.periodic_warp(X, L, 0.05)


def _pair(n, N, dt, mu=None, features=0, vel=None):
    from paper_1704_04549_gb300 import Context
    vel = vel or synthetic.fourier_velocity(1705, 2)
    h = L / N
    ctx = Context(2, n, (N, N), h, dt, vel, features=features, device=DEV, mu=mu or 0)
    jd, fl, ff = mesh.warped_metric_terms((N, N), h, ctx.gauss_legendre()[0], vel, _warp)
    ctx.tpp_set_metric_terms(jd, fl, ff, dt)
    return ctx, CurvedAdvectionDG(PeriodicMesh((N, N), h), n, dt, vel, _warp, mu)


CASES = [(2, 3, None), (5, 3, None), (8, 4, None), (16, 2, None), (31, 2, None),
         (4, 3, 7), (8, 3, 12), (16, 2, 24)]


@pytest.mark.parametrize("n,N,mu", CASES)
def test_curved_operator_matches_oracle(n, N, mu):
    ctx, ora = _pair(n, N, 0.05, mu)
    S = ora.global_matrix()
    x = synthetic.rhs(7, ora.ndof)
    y = to_host(ctx.dg_apply_sumfact(to_dev(x)))
    assert rel(y, S @ x) <= FP64_TOL, rel(y, S @ x)
    if n <= 16:
        ys = to_host(ctx.dg_apply_sumfact_static(to_dev(x)))
        assert rel(ys, S @ x) <= FP64_TOL


@pytest.mark.parametrize("n,N,mu", [c for c in CASES if c[0] <= 16])
@pytest.mark.parametrize("form", ["one-sided", "two-sided"])
def test_curved_factors_and_apply(n, N, mu, form):
    ctx, ora = _pair(n, N, 0.05, mu, features=TPP_FEAT_TWO_SIDED if form == "two-sided" else 0)
    rep = ctx.tpp_build_factors()
    assert rep["num_schur_fail"] == 0
    _check_elements(ctx, ora, list(range(ora.mesh.num_elem)))


@pytest.mark.parametrize("n,N", [(4, 3), (8, 3)])
def test_curved_block_jacobi(n, N):
    ctx, ora = _pair(n, N, 0.05, features=TPP_FEAT_BLOCK_JACOBI)
    ctx.tpp_build_block_jacobi()
    b = synthetic.rhs(5, ora.ndof)
    x = to_host(ctx.tpp_apply_block_jacobi(to_dev(b)))
    nl = ora.nloc
    for e in range(ora.mesh.num_elem):
        Se = ora.element_block(e)
        ref = np.linalg.solve(Se, b[e * nl:(e + 1) * nl])
        assert rel(x[e * nl:(e + 1) * nl], ref) <= FP64_TOL * np.linalg.cond(Se)


@pytest.mark.parametrize("n,N,mu", [(5, 4, None), (8, 4, None), (6, 3, 9)])
def test_curved_gmres_matches_oracle(n, N, mu):
    ctx, ora = _pair(n, N, 0.05, mu)
    ctx.tpp_build_factors()
    S = ora.global_matrix()
    b = synthetic.rhs(1706, ora.ndof)
    x_ref, o = gmres(lambda v: S @ v, b, M=kron_dense(ora), rtol=1e-8)
    assert o["converged"]
    x, r = ctx.gmres_solve(to_dev(b), pc=TPP_PC_KRON, rtol=1e-8)
    assert r["converged"] and r["true_rel_res"] <= 1e-8
    assert abs(r["iters"] - o["iters"]) <= 1
    assert rel(to_host(x), spla.spsolve(S.tocsc(), b)) <= 1e-6


def test_curved_mixed_precision():
    """FP32 operator (per-point mass in float) and the nested mixed solver."""
    ctx, ora = _pair(8, 4, 0.05, features=TPP_FEAT_MIXED)
    ctx.tpp_build_factors()
    S = ora.global_matrix()
    v = synthetic.rhs(11, ora.ndof)
    y32 = to_host(ctx.dg_apply_sumfact_f32(torch.as_tensor(v.astype(np.float32), device=DEV)))
    err = rel(y32.astype(np.float64), S @ v.astype(np.float32).astype(np.float64))
    print(f"FP32 curved operator: relative error {err:.2e}")
    assert err <= 1e-5
    b = synthetic.rhs(12, ora.ndof)
    x, r = ctx.gmres_solve(to_dev(b), pc=TPP_PC_KRON, rtol=1e-10, inner_iters=8)
    assert r["converged"] and np.linalg.norm(b - S @ to_host(x)) <= 1.0001e-10 * np.linalg.norm(b)


def test_set_velocity_returns_to_affine_elements():
    vel = synthetic.fourier_velocity(1705, 2)
    ctx, _ = _pair(6, 3, 0.05, vel=vel)
    vn, fn = mesh.periodic_field((3, 3), ctx.gauss_legendre()[0], vel)
    ctx.tpp_set_velocity(vn, fn, 0.05)
    aff = AdvectionDG(PeriodicMesh((3, 3), L / 3), 6, 0.05, vel).global_matrix()
    x = synthetic.rhs(3, ctx.num_dofs)
    assert rel(to_host(ctx.dg_apply_sumfact(to_dev(x))), aff @ x) <= FP64_TOL
