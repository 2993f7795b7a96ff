"""GPU parity: over-integration (mu > n quadrature points per direction, Sec. 3.2
and Sec. 4.2) vs the oracle.  The operator is checked against the assembled
matrix, the KSVD factors of the explicit over-integrated cores against the
oracle's rearrangement SVD of the dense block, and GMRES against the oracle's
preconditioned GMRES."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla
import torch

import synthetic
from oracle.gmres import gmres
from oracle.precond import kron_dense
from paper_1704_04549_gb300 import TPP_FEAT_MIXED, TPP_FEAT_TWO_SIDED, TPP_PC_KRON
from tests.gpu_util import DEV, FP64_TOL, make_pair, rel, to_dev, to_host
from tests.test_gpu_factors import _check_elements

pytestmark = pytest.mark.gpu

# (n, mu, mesh): mu = n + 1 and the usual 3n/2 rule, odd n with odd mu (the points
# coincide with a node at 1/2), small n where 2 mu + 2 > n^2 (core = full n^2 space),
# and the largest mu
CASES = [(2, 3, (3, 2)), (3, 5, (3, 3)), (4, 6, (3, 4)), (5, 7, (3, 5)), (8, 12, (4, 4)),
         (8, 9, (3, 3)), (16, 24, (3, 3)), (16, 32, (2, 3)), (31, 32, (2, 2))]


@pytest.mark.parametrize("n,mu,nel", CASES)
def test_quadrature_rule_and_operator(n, mu, nel):
    ctx, dg = make_pair(n, nel, 0.05, synthetic.fourier_velocity(1705, 2), mu=mu)
    x, w = ctx.gauss_legendre()
    assert np.allclose(x, dg.basis.x, rtol=0, atol=2e-16)
    assert np.allclose(w, dg.basis.w, rtol=1e-13, atol=0)
    S = dg.global_matrix()
    v = synthetic.rhs(7, dg.ndof)
    y = to_host(ctx.dg_apply_sumfact(to_dev(v)))
    assert rel(y, S @ v) <= FP64_TOL, rel(y, S @ v)
    ys = to_host(ctx.dg_apply_sumfact_static(to_dev(v)))
    assert rel(ys, S @ v) <= FP64_TOL


@pytest.mark.parametrize("n,mu,nel", CASES)
@pytest.mark.parametrize("form", ["one-sided", "two-sided"])
def test_factors_and_apply(n, mu, nel, form):
    ctx, dg = make_pair(n, nel, 0.05, synthetic.fourier_velocity(1705, 2), mu=mu,
                        features=TPP_FEAT_TWO_SIDED if form == "two-sided" else 0)
    rep = ctx.tpp_build_factors()
    assert rep["num_schur_fail"] == 0
    _check_elements(ctx, dg, list(range(dg.mesh.num_elem)))


def test_over_integration_changes_the_operator():
    """The mu > n operator is not the collocated one (the aliasing terms differ), and
    on a constant field it still matches the assembled over-integrated matrix."""
    vel = synthetic.fourier_velocity(1705, 2)
    c0, d0 = make_pair(6, (3, 3), 0.05, vel)
    c1, d1 = make_pair(6, (3, 3), 0.05, vel, mu=9)
    v = synthetic.rhs(4, d0.ndof)
    y0, y1 = to_host(c0.dg_apply_sumfact(to_dev(v))), to_host(c1.dg_apply_sumfact(to_dev(v)))
    assert rel(y1, y0) > 1e-6
    one = np.ones(d1.ndof)
    y = to_host(c1.dg_apply_sumfact(to_dev(one)))
    assert rel(y, d1.global_matrix() @ one) <= FP64_TOL


@pytest.mark.parametrize("n,mu,nel", [(5, 8, (4, 4)), (8, 12, (4, 4)), (12, 18, (4, 4))])
def test_gmres_matches_oracle(n, mu, nel):
    ctx, dg = make_pair(n, nel, 0.05, synthetic.fourier_velocity(1705, 2), mu=mu, h=1.0)
    ctx.tpp_build_factors()
    b = synthetic.rhs(1706, dg.ndof)
    S = dg.global_matrix()
    x_ref, o = gmres(lambda v: S @ v, b, M=kron_dense(dg), rtol=1e-8)
    assert o["converged"]
    x, r = ctx.gmres_solve(to_dev(b), pc=TPP_PC_KRON, rtol=1e-8)
    assert r["converged"] and r["true_rel_res"] <= 1e-8
    assert abs(r["iters"] - o["iters"]) <= 1
    assert rel(to_host(x), x_ref) <= 1e-6
    x12, r12 = ctx.gmres_solve(to_dev(b), pc=TPP_PC_KRON, rtol=1e-12)
    assert r12["true_rel_res"] <= 1e-12
    assert rel(to_host(x12), spla.spsolve(S.tocsc(), b)) <= 1e-9


def test_mixed_precision_operator_and_solve():
    """FP32 operator and FP32 inner preconditioner on the over-integrated problem."""
    n, mu = 8, 12
    ctx, dg = make_pair(n, (4, 4), 0.05, synthetic.fourier_velocity(1705, 2), mu=mu,
                        features=TPP_FEAT_MIXED, h=1.0)
    ctx.tpp_build_factors()
    S = dg.global_matrix()
    v = synthetic.rhs(11, dg.ndof)
    y32 = to_host(ctx.dg_apply_sumfact_f32(torch.as_tensor(v.astype(np.float32), device=DEV)))
    # norm-wise: every output sums about 2 (n + mu) + 10 rounded FP32 products; 1e-5
    # is about 84 u32 (the measured error is printed)
    err = rel(y32.astype(np.float64), S @ v.astype(np.float32).astype(np.float64))
    print(f"FP32 over-integrated operator, n={n} mu={mu}: relative error {err:.2e}")
    assert err <= 1e-5
    b = synthetic.rhs(12, dg.ndof)
    x, r = ctx.gmres_solve(to_dev(b), pc=TPP_PC_KRON, rtol=1e-10, inner_iters=8)
    assert r["converged"] and r["true_rel_res"] <= 1e-10
    assert np.linalg.norm(b - S @ to_host(x)) <= 1.0001e-10 * np.linalg.norm(b)
