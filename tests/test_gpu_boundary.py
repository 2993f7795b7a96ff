"""GPU: the problem description of the C ABI (tpp_problem: velocity at the nodes,
a.n at the faces, the neighbour table, right-hand sides per element) exercised
beyond the Cartesian numbering, against the oracle."""
import numpy as np
import pytest
import torch

import synthetic
from oracle.dg import AdvectionDG, PeriodicMesh
from oracle.ksvd import ksvd_2d, kron_sum
from oracle.precond import apply_dense
from paper_1704_04549_gb300 import TPP_PC_KRON, Context, mesh
from tests.gpu_util import DEV, rel, solve_tol, to_dev, to_host

pytestmark = pytest.mark.gpu


def _arrays(nel, n, vel):
    """Neighbour table and field arrays of the periodic mesh (element order ex + N ey)."""
    ctx = Context(len(nel), n, nel, 1.0, 0.05, vel, device=DEV)
    x = ctx.gauss_legendre()[0]
    return (mesh.periodic_nbr(nel),) + mesh.periodic_field(nel, x, vel)


def test_renumbered_elements_match_oracle():
    """The periodic 4 x 5 mesh with its elements renumbered by a random permutation
    (so neighbours are found only through nbr): operator, preconditioner apply and
    GMRES equal the oracle's on the permuted blocks."""
    nel, n, dim = (4, 5), 5, 2
    vel = synthetic.fourier_velocity(1705, 2)
    nbr, vn, fn = _arrays(nel, n, vel)
    E, nl = nbr.shape[0], n * n
    perm = np.random.Generator(np.random.PCG64(5)).permutation(E)     # new id of element e
    inv = np.argsort(perm)                                            # old id of new element
    nbr2 = perm[nbr[inv]].astype(np.int32)
    vn2 = vn.reshape(dim, E, nl)[:, inv].reshape(dim, -1)
    fn2 = fn[inv]
    ctx = Context.from_arrays(dim, n, 1.0, 0.05, nbr2, vn2, fn2, device=DEV)
    dg = AdvectionDG(PeriodicMesh(nel, 1.0), n, 0.05, vel)
    S = dg.global_matrix()
    b = synthetic.rhs(11, dg.ndof)
    b2 = b.reshape(E, nl)[inv].reshape(-1)
    y2 = to_host(ctx.dg_apply_sumfact(to_dev(b2)))
    y = S @ b
    assert rel(y2, y.reshape(E, nl)[inv].reshape(-1)) <= 1e-13
    ctx.tpp_build_factors()
    x2 = to_host(ctx.tpp_apply_inverse(to_dev(b2))).reshape(E, nl)
    for e_new in range(E):
        _, As, Bs = ksvd_2d(dg.element_block(inv[e_new]), n)
        P = kron_sum(As, Bs)
        x_ref = apply_dense(P, b.reshape(E, nl)[inv[e_new]])
        assert rel(x2[e_new], x_ref) <= solve_tol(np.linalg.cond(P))
    ctx0 = Context(dim, n, nel, 1.0, 0.05, vel, device=DEV)
    ctx0.tpp_build_factors()
    _, r0 = ctx0.gmres_solve(to_dev(b), pc=TPP_PC_KRON, rtol=1e-10)
    xs, r2 = ctx.gmres_solve(to_dev(b2), pc=TPP_PC_KRON, rtol=1e-10)
    assert r2["converged"] and abs(r2["iters"] - r0["iters"]) <= 1
    xs = to_host(xs).reshape(E, nl)[perm].reshape(-1)          # back to the original order
    assert np.linalg.norm(S @ xs - b) <= 1.0001e-10 * np.linalg.norm(b)


@pytest.mark.parametrize("dim,nel,n", [(2, (3, 4), 6), (3, (2, 3, 2), 4)])
def test_several_right_hand_sides_on_a_mesh(dim, nel, n):
    """nrhs = 3 right-hand sides per element on a coupled periodic mesh (vectors
    [E][3][n^d], the inflow of a face read from the neighbour's same right-hand side):
    each right-hand side matches the oracle's operator; a call on the first
    right-hand side alone (per-call nrhs = 1) matches too; the preconditioner acts per
    right-hand side; GMRES solves all three at once."""
    vel = synthetic.fourier_velocity(1705, dim)
    nbr, vn, fn = _arrays(nel, n, vel)
    E, nl, R = nbr.shape[0], n ** dim, 3
    ctx = Context.from_arrays(dim, n, 1.0, 0.05, nbr, vn, fn, nrhs=R, device=DEV)
    dg = AdvectionDG(PeriodicMesh(nel, 1.0), n, 0.05, vel)
    S = dg.global_matrix()
    B = synthetic.rhs(12, E * R * nl).reshape(E, R, nl)
    Y = to_host(ctx.dg_apply_sumfact(to_dev(B.reshape(-1)))).reshape(E, R, nl)
    for r in range(R):
        assert rel(Y[:, r].reshape(-1), S @ B[:, r].reshape(-1)) <= 1e-13
    y0 = to_host(ctx.dg_apply_sumfact(to_dev(B[:, 0].reshape(-1)), nrhs=1))
    assert rel(y0, Y[:, 0].reshape(-1)) <= 1e-15
    ctx.tpp_build_factors()
    X = to_host(ctx.tpp_apply_inverse(to_dev(B.reshape(-1)))).reshape(E, R, nl)
    x1 = to_host(ctx.tpp_apply_inverse(to_dev(B[:, 1].reshape(-1)), nrhs=1)).reshape(E, nl)
    assert np.array_equal(x1, X[:, 1])
    xs, res = ctx.gmres_solve(to_dev(B.reshape(-1)), pc=TPP_PC_KRON, rtol=1e-10)
    assert res["converged"]
    Xs = to_host(xs).reshape(E, R, nl)
    for r in range(R):
        br = B[:, r].reshape(-1)
        assert np.linalg.norm(S @ Xs[:, r].reshape(-1) - br) <= 1e-9 * np.linalg.norm(br)
    with pytest.raises(Exception):
        ctx.dg_apply_sumfact(to_dev(np.zeros(E * 4 * nl)), nrhs=4)


def test_set_velocity_matches_a_fresh_context():
    """tpp_set_velocity (a new field and step on an existing context) gives the
    operator and the factors of a context created with them, bit for bit."""
    nel, n = (4, 4), 7
    v1, v2 = synthetic.fourier_velocity(3, 2), synthetic.fourier_velocity(4, 2)
    ctx = Context(2, n, nel, 1.0, 0.05, v1, device=DEV)
    ctx.tpp_build_factors()
    x = ctx.gauss_legendre()[0]
    vn, fn = mesh.periodic_field(nel, x, v2)
    ctx.tpp_set_velocity(vn, fn, 0.08)
    ref = Context(2, n, nel, 1.0, 0.08, v2, device=DEV)
    b = to_dev(synthetic.rhs(13, ref.num_dofs))
    assert torch.equal(ctx.dg_apply_sumfact(b), ref.dg_apply_sumfact(b))
    with pytest.raises(Exception):
        ctx.tpp_apply_inverse(b)                 # the old factors are stale
    ctx.tpp_build_factors()
    ref.tpp_build_factors()
    assert torch.equal(ctx.tpp_apply_inverse(b), ref.tpp_apply_inverse(b))
    dg = AdvectionDG(PeriodicMesh(nel, 1.0), n, 0.08, v2)
    assert rel(to_host(ctx.dg_apply_sumfact(b)), dg.global_matrix() @ to_host(b)) <= 1e-13
