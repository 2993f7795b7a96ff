"""GPU parity: KSVD factor build and preconditioner apply vs the oracle."""
import numpy as np
import pytest

import synthetic
from oracle.ksvd import ksvd_2d, kron_sum
from oracle.precond import apply_dense
from paper_1704_04549_gb300 import TPP_FEAT_TWO_SIDED
from tests.gpu_util import FP64_TOL, make_pair, rel, solve_tol, to_dev, to_host

pytestmark = pytest.mark.gpu


def _check_elements(ctx, dg, elems, tol_sigma=FP64_TOL, tol_P=FP64_TOL, tol_x=FP64_TOL):
    v = ctx.views()
    sig = to_host(v["sigma"])
    A1, B1, A2, B2 = (to_host(v[k]) for k in ("A1", "B1", "A2", "B2"))
    flags = to_host(v["flags"])
    cpair = to_host(v["cond"])
    n, nl = dg.n, dg.nloc
    b = synthetic.rhs(99, dg.ndof)
    x = to_host(ctx.tpp_apply_inverse(to_dev(b)))
    worst = 0.0
    for e in elems:
        S = dg.element_block(e)
        s_ref, As, Bs = ksvd_2d(S, n)
        P_ref = kron_sum(As, Bs)
        assert abs(sig[e, 0] - s_ref[0]) <= tol_sigma * s_ref[0]
        if n > 1:
            assert abs(sig[e, 1] - s_ref[1]) <= tol_sigma * s_ref[0]
        P = np.kron(A1[e], B1[e]) + np.kron(A2[e], B2[e])
        assert rel(P, P_ref) <= tol_P, (e, rel(P, P_ref))
        be = b[e * nl:(e + 1) * nl]
        x_ref = apply_dense(P_ref, be)
        err = rel(x[e * nl:(e + 1) * nl], x_ref)
        kappa = np.linalg.cond(P_ref)
        worst = max(worst, err)
        assert err <= max(tol_x, solve_tol(kappa, cpair[e])), (e, err, kappa, cpair[e])
        assert cpair[e] <= 1e8, (e, cpair[e])
        assert flags[e] & 12 == 0          # no Schur failure, no singular factor
    print(f"FP64 apply vs oracle, n={n}: max element relative error {worst:.2e} "
          f"over {len(elems)} elements")


@pytest.mark.parametrize("n,nel,field", [(2, (3, 2), "fourier"), (3, (3, 3), "fourier"),
                                         (5, (3, 5), "fourier"), (8, (8, 8), "const"),
                                         (8, (4, 4), "fourier"), (16, (3, 3), "fourier"),
                                         (31, (2, 2), "fourier"), (32, (1, 2), "fourier")])
@pytest.mark.parametrize("form", ["one-sided", "two-sided"])
def test_factors_and_apply_match_oracle(n, nel, field, form):
    vel = (synthetic.constant_velocity([1.0, 0.5]) if field == "const"
           else synthetic.fourier_velocity(1705, 2))
    ctx, dg = make_pair(n, nel, 0.05, vel,
                        features=TPP_FEAT_TWO_SIDED if form == "two-sided" else 0)
    rep = ctx.tpp_build_factors()
    assert rep["num_schur_fail"] == 0
    elems = list(range(dg.mesh.num_elem)) if dg.mesh.num_elem <= 16 else [0, 5, dg.mesh.num_elem - 1]
    _check_elements(ctx, dg, elems)


def test_rank_one_limit_dt_zero():
    """dt = 0: the block is the mass matrix h^2 W (x) W, a single Kronecker product."""
    n = 6
    ctx, dg = make_pair(n, (2, 2), 0.0, synthetic.fourier_velocity(3, 2))
    rep = ctx.tpp_build_factors()
    assert rep["num_rank1"] == 4
    b = synthetic.rhs(5, dg.ndof)
    x = to_host(ctx.tpp_apply_inverse(to_dev(b)))
    w = dg.basis.w
    m = np.tile(dg.mesh.h ** 2 * np.outer(w, w).reshape(-1), 4)
    assert rel(x, b / m) <= 1e-13


def test_n1_finite_volume():
    ctx, dg = make_pair(1, (4, 4), 0.1, synthetic.fourier_velocity(8, 2))
    ctx.tpp_build_factors()
    b = synthetic.rhs(3, dg.ndof)
    x = to_host(ctx.tpp_apply_inverse(to_dev(b)))
    d = np.array([dg.element_block(e)[0, 0] for e in range(16)])
    assert rel(x, b / d) <= 1e-14


def test_exact_recovery_constant_velocity_full_size():
    """64 x 64, n = 16, constant velocity: sigma_3 = 0 so P equals the exact block."""
    n = 16
    ctx, dg = make_pair(n, (64, 64), 0.05, synthetic.constant_velocity([1.0, 0.5]))
    ctx.tpp_build_factors()
    v = ctx.views()
    A1, B1, A2, B2 = (to_host(v[k]) for k in ("A1", "B1", "A2", "B2"))
    for e in [0, 1000, 4095]:
        S = dg.element_block(e)
        P = np.kron(A1[e], B1[e]) + np.kron(A2[e], B2[e])
        assert rel(P, S) <= 1e-13


@pytest.mark.parametrize("n,h", [(16, 1.0), (31, 1.0), (31, 1.0 / 64)])
def test_full_size_sampled_elements(n, h):
    """64 x 64 periodic mesh with the random-Fourier field: sampled elements."""
    ctx, dg = make_pair(n, (64, 64), 0.05, synthetic.fourier_velocity(1705, 2), h=h)
    rep = ctx.tpp_build_factors()
    assert rep["num_schur_fail"] == 0
    _check_elements(ctx, dg, [0, 2049, 4095] if n == 16 else [17, 712, 3000, 3785])
