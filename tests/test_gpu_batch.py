"""GPU parity in batch mode: block-diagonal systems of isolated elements with
several right-hand sides each (the mixed-degree batch, one degree group per
context), against the oracle's isolated-element blocks."""
import numpy as np
import pytest
import scipy.linalg as sla
import torch

import synthetic
from oracle.dg import IsolatedElements
from oracle.ksvd import kron_sum, ksvd_2d, ksvd_3d_nested
from oracle.precond import apply_dense
from paper_1704_04549_gb300 import TPP_FEAT_MIXED, TPP_PC_KRON
from tests.gpu_util import DEV, rel, solve_tol, to_dev, to_host

pytestmark = pytest.mark.gpu

H, DT = 1.0 / 64, 0.05


def _batch(dim, n, E, R, seed=5, h=H, span=H):
    from paper_1704_04549_gb300 import Context
    rng = np.random.Generator(np.random.PCG64(seed))
    centres = rng.random((E, dim))
    vel = synthetic.fourier_velocity(1709, dim)
    ctx = Context(dim, n, (E,), h, DT, vel, features=TPP_FEAT_MIXED, device=DEV,
                  batch_rhs=R, centres=centres, batch_span=span)
    return ctx, IsolatedElements(n, h, centres, DT, vel, span=span)


# (dim, n, elements, right-hand sides, element width); h = 1: unit elements sampling
# 1/64 of the field (the batch workload's reading), h = 1/64: elements of the unit domain
CASES = [(2, 1, 3, 2, H), (2, 5, 7, 3, H), (2, 16, 4, 2, H), (2, 31, 2, 2, H), (3, 3, 5, 2, H),
         (3, 6, 3, 3, H), (2, 16, 5, 2, 1.0), (3, 11, 2, 2, 1.0)]


@pytest.mark.parametrize("dim,n,E,R,h", CASES)
def test_batch_operator_matches_isolated_blocks(dim, n, E, R, h):
    ctx, iso = _batch(dim, n, E, R, h=h)
    nl = iso.nloc
    x = synthetic.rhs(3, E * R * nl)
    y = to_host(ctx.dg_apply_sumfact(to_dev(x))).reshape(E, R, nl)
    X = x.reshape(E, R, nl)
    for e in range(E):
        S = iso.block(e)
        for r in range(R):
            assert rel(y[e, r], S @ X[e, r]) <= 1e-12


@pytest.mark.parametrize("dim,n,E,R,h", CASES)
def test_batch_factors_and_apply_match_oracle(dim, n, E, R, h):
    ctx, iso = _batch(dim, n, E, R, h=h)
    rep = ctx.tpp_build_factors()
    assert rep["num_schur_fail"] == 0
    nl = iso.nloc
    b = synthetic.rhs(4, E * R * nl)
    x = to_host(ctx.tpp_apply_inverse(to_dev(b))).reshape(E, R, nl)
    B = b.reshape(E, R, nl)
    v = ctx.views()
    cpair = to_host(v["cond"])
    for e in range(E):
        S = iso.block(e)
        if dim == 2:
            _, As, Bs = ksvd_2d(S, n)
            P = kron_sum(As, Bs)
            cz = 1.0
        else:
            P = ksvd_3d_nested(S, n)["P"]
            cz = np.linalg.cond(to_host(v["Az"])[e], 1)
        kappa = np.linalg.cond(P)
        for r in range(R):
            err = rel(x[e, r], apply_dense(P, B[e, r]))
            assert err <= solve_tol(kappa, cpair[e] * cz), (e, r, err, kappa, cpair[e], cz)


@pytest.mark.parametrize("dim,n,E,R,h", [(2, 8, 12, 4, H), (2, 16, 6, 3, 1.0), (2, 31, 3, 2, 1.0),
                                          (3, 5, 6, 2, H), (3, 11, 3, 2, 1.0)])
def test_batch_gmres_solves_every_block(dim, n, E, R, h):
    """One Krylov solve of the whole block-diagonal system, FP64 and nested mixed."""
    ctx, iso = _batch(dim, n, E, R, h=h)
    ctx.tpp_build_factors()
    nl = iso.nloc
    b = synthetic.rhs(6, E * R * nl)
    B = b.reshape(E, R, nl)
    ref = np.stack([np.stack([sla.solve(iso.block(e), B[e, r]) for r in range(R)])
                    for e in range(E)])
    for kw in (dict(), dict(inner_iters=12)):
        x, res = ctx.gmres_solve(to_dev(b), pc=TPP_PC_KRON, rtol=1e-8, **kw)
        assert res["converged"] and res["true_rel_res"] <= 1e-8
        assert rel(to_host(x).reshape(E, R, nl), ref) <= 1e-6
