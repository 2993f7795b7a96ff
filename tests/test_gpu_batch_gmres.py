"""GPU parity: per-system batched GMRES (tpp_batch_gmres) over a mixed-degree batch
of isolated elements, against the oracle.  Every (element, right-hand side) system
is checked on its own: its true relative residual with the oracle's block, its
solution against a dense solve of the block, and (FP64) its Arnoldi step count
against the oracle's GMRES with the oracle's Kronecker preconditioner."""
import numpy as np
import pytest
import scipy.linalg as sla

import synthetic
from oracle.dg import IsolatedElements
from oracle.gmres import gmres
from oracle.ksvd import kron_sum, ksvd_2d, ksvd_3d_nested
from paper_1704_04549_gb300 import TPP_FEAT_MIXED, TPP_FEAT_TWO_SIDED
from paper_1704_04549_gb300._lib import TppError
from tests.gpu_util import DEV, rel, to_dev, to_host

pytestmark = pytest.mark.gpu

DT, R, RESTART = 0.05, 3, 20
# (dim, n, elements): every lane-group width (8, 16, 32), odd and even n, 2D and 3D
GROUPS = [(2, 2, 3), (2, 5, 4), (2, 8, 3), (2, 12, 3), (2, 17, 2), (2, 31, 2),
          (3, 3, 3), (3, 8, 2), (3, 11, 2)]


def _group(dim, n, E, seed, mixed, h=1.0, span=1.0 / 64):
    from paper_1704_04549_gb300 import Context
    rng = np.random.Generator(np.random.PCG64(seed))
    centres = rng.random((E, dim))
    vel = synthetic.fourier_velocity(1709, dim)
    feats = TPP_FEAT_TWO_SIDED | (TPP_FEAT_MIXED if mixed else 0)
    ctx = Context(dim, n, (E,), h, DT, vel, features=feats, device=DEV, batch_rhs=R,
                  centres=centres, batch_span=span)
    ctx.tpp_build_factors()
    return ctx, IsolatedElements(n, h, centres, DT, vel, span=span)


def _batch(mixed, groups=GROUPS):
    ctxs, isos, bs, xs = [], [], [], []
    for k, (dim, n, E) in enumerate(groups):
        ctx, iso = _group(dim, n, E, 40 + k, mixed)
        b = synthetic.rhs(50 + k, E * R * iso.nloc)
        ctxs.append(ctx)
        isos.append(iso)
        bs.append(to_dev(b))
        xs.append(to_dev(np.zeros_like(b)))
    return ctxs, isos, bs, xs


def _oracle_P(iso, e):
    S = iso.block(e)
    if iso.dim == 2:
        _, As, Bs = ksvd_2d(S, iso.n)
        return S, kron_sum(As, Bs)
    return S, ksvd_3d_nested(S, iso.n)["P"]


@pytest.mark.parametrize("mixed", [False, True])
def test_every_system_converges_to_the_oracle_solution(mixed):
    from paper_1704_04549_gb300.batch import BatchGmres
    ctxs, isos, bs, xs = _batch(mixed)
    solver = BatchGmres(ctxs, restart=RESTART, rtol=1e-8, max_iters=400, mixed=mixed,
                        inner_rtol=1e-4, max_outer=8, per_system=True)
    rep = solver.solve(bs, xs)
    assert rep["unconverged"] == 0 and rep["max_relres"] <= 1e-8
    assert rep["systems"] == sum(E * R for _, _, E in GROUPS)
    assert rep["launches"] == 3
    worst_res = worst_x = 0.0
    iter_diff = []
    for g, (ctx, iso) in enumerate(zip(ctxs, isos)):
        nl = iso.nloc
        E = iso.num_elem
        x = to_host(xs[g]).reshape(E, R, nl)
        b = to_host(bs[g]).reshape(E, R, nl)
        its = to_host(solver.iters[g]).reshape(E, R)
        rr = to_host(solver.relres[g]).reshape(E, R)
        for e in range(E):
            S, P = _oracle_P(iso, e)
            Pinv = np.linalg.inv(P)
            for r in range(R):
                res = np.linalg.norm(b[e, r] - S @ x[e, r]) / np.linalg.norm(b[e, r])
                assert rr[e, r] <= 1e-8 and res <= 1.01e-8, (g, e, r, res, rr[e, r])
                err = rel(x[e, r], sla.solve(S, b[e, r]))
                assert err <= 1e-6, (g, e, r, err)
                worst_res, worst_x = max(worst_res, res), max(worst_x, err)
                if not mixed:
                    _, o = gmres(lambda v: S @ v, b[e, r], M=lambda v: Pinv @ v,
                                 restart=RESTART, rtol=1e-8)
                    assert o["converged"]
                    iter_diff.append(abs(int(its[e, r]) - o["iters"]))
    if not mixed:
        assert max(iter_diff) <= 1, iter_diff
    print(f"batched GMRES ({'mixed' if mixed else 'FP64'}): {rep['systems']} systems, "
          f"{rep['total_iters']} Arnoldi steps, max {rep['max_iters']}, worst true residual "
          f"{worst_res:.2e}, worst solution error {worst_x:.2e}")


def test_second_solve_reuses_the_workspace():
    """Two solves in a row with one BatchGmres give the same iterates (no state is
    carried between calls: queues, counters and statistics restart)."""
    from paper_1704_04549_gb300.batch import BatchGmres
    groups = [(2, 6, 3), (2, 20, 2), (3, 5, 2)]
    ctxs, isos, bs, xs = _batch(False, groups)
    solver = BatchGmres(ctxs, restart=RESTART, rtol=1e-8)
    r1 = solver.solve(bs, xs)
    first = [to_host(x).copy() for x in xs]
    for x in xs:
        x.fill_(123.0)
    r2 = solver.solve(bs, xs)
    assert r1["total_iters"] == r2["total_iters"] and r1["max_iters"] == r2["max_iters"]
    for a, x in zip(first, xs):
        assert np.array_equal(a, to_host(x))


def test_invalid_contexts_and_options_are_rejected():
    from paper_1704_04549_gb300 import Context
    from paper_1704_04549_gb300.batch import BatchGmres
    good = _group(2, 6, 2, 3, False)[0]
    coupled = Context(2, 6, (3, 3), 1.0 / 3, DT, synthetic.fourier_velocity(1705, 2),
                      features=TPP_FEAT_TWO_SIDED, device=DEV)
    plain = Context(2, 6, (2,), 1.0, DT, synthetic.fourier_velocity(1709, 2), device=DEV,
                    batch_rhs=2, centres=np.array([[0.2, 0.3], [0.6, 0.7]]),
                    batch_span=1.0 / 64)
    with pytest.raises(TppError, match="isolated"):
        BatchGmres([coupled])
    with pytest.raises(TppError, match="TWO_SIDED"):
        BatchGmres([plain])
    with pytest.raises(TppError, match="restart"):
        BatchGmres([good], restart=40)
    with pytest.raises(TppError, match="TPP_FEAT_MIXED"):
        BatchGmres([good], mixed=True)


@pytest.mark.parametrize("mixed", [False, True])
def test_launch_shapes_give_identical_results(mixed):
    """Warps per CTA, CTAs per SM and the register budget (the autotuner's choices) change
    only the schedule: every system's iterate is bit-identical across shapes."""
    from paper_1704_04549_gb300.batch import BatchGmres
    groups = [(2, 4, 3), (2, 13, 2), (2, 25, 2), (3, 6, 2)]
    ctxs, isos, bs, xs = _batch(mixed, groups)
    ref = None
    for w, c, rb in [(8, 0, 1), (2, 1, 2), (4, 0, 2), (8, 1, 1)]:
        solver = BatchGmres(ctxs, restart=RESTART, rtol=1e-8, mixed=mixed, warps=(w,) * 3,
                            ctas_per_sm=(c,) * 3, reg_budget=(rb,) * 3)
        rep = solver.solve(bs, xs)
        assert rep["unconverged"] == 0 and all(t > 0 for t in rep["launch_ms"])
        got = [to_host(x).copy() for x in xs]
        if ref is None:
            ref = got
        else:
            assert all(np.array_equal(a, b) for a, b in zip(ref, got)), (w, c, rb)
