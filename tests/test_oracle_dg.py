"""Pins for oracle/dg.py against closed forms, exact integrals and invariants."""
import numpy as np
import pytest

import synthetic
from oracle.dg import AdvectionDG, PeriodicMesh


def _exact_1d(n):
    """Exact 1D mass, stiffness and endpoint values of the Lagrange basis on the
    Gauss-Legendre nodes, computed in a Legendre-series representation (an
    independent route: interpolation by a Legendre Vandermonde, exact series
    products and antiderivatives)."""
    import numpy.polynomial.legendre as L
    from oracle.basis import gauss_legendre_01
    nodes, _ = gauss_legendre_01(n)
    t = 2.0 * nodes - 1.0                       # [0,1] -> [-1,1]
    C = np.linalg.solve(L.legvander(t, n - 1), np.eye(n)).T   # row j: phi_j in Legendre series
    m = np.zeros((n, n))
    c = np.zeros((n, n))
    for i in range(n):
        for k in range(n):
            pik = L.legint(L.legmul(C[i], C[k]))
            m[i, k] = 0.5 * (L.legval(1.0, pik) - L.legval(-1.0, pik))      # dx = dt/2
            dik = L.legint(L.legmul(2.0 * L.legder(C[i]), C[k]))           # d/dx = 2 d/dt
            c[i, k] = 0.5 * (L.legval(1.0, dik) - L.legval(-1.0, dik))
    l0 = np.array([L.legval(-1.0, C[j]) for j in range(n)])
    l1 = np.array([L.legval(1.0, C[j]) for j in range(n)])
    return m, c, l0, l1


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 12])
def test_block_equals_exact_integrals_constant_velocity(n):
    ax, ay, h, dt = 0.7, -1.3, 0.25, 0.2
    dg = AdvectionDG(PeriodicMesh((4, 4)), n, dt, synthetic.constant_velocity([ax, ay]))
    m, c, l0, l1 = _exact_1d(n)
    pos, neg = lambda v: max(v, 0.0), lambda v: min(v, 0.0)
    S = (h * h * np.kron(m, m)
         - dt * h * (ax * np.kron(m, c) + ay * np.kron(c, m))
         + dt * h * (pos(ax) * np.kron(m, np.outer(l1, l1)) + pos(-ax) * np.kron(m, np.outer(l0, l0))
                     + pos(ay) * np.kron(np.outer(l1, l1), m) + pos(-ay) * np.kron(np.outer(l0, l0), m)))
    e = 5
    assert np.allclose(dg.element_block(e), S, rtol=0, atol=1e-12 * np.abs(S).max())
    _, nbrs = dg.face_blocks(e)
    # -x neighbour (left element) enters through its +x trace
    nb, F = nbrs[0]
    assert nb == dg.mesh.index((0, 1))
    assert np.allclose(F, h * neg(-ax) * np.kron(m, np.outer(l0, l1)), atol=1e-13)
    nb, F = nbrs[3]      # +y neighbour, inflow since ay < 0
    assert np.allclose(F, h * neg(ay) * np.kron(np.outer(l1, l0), m), atol=1e-13)


def test_n1_is_first_order_upwind_finite_volume():
    ax, ay, h, dt = 1.0, 0.5, 1 / 8, 0.1
    dg = AdvectionDG(PeriodicMesh((8, 8)), 1, dt, synthetic.constant_velocity([ax, ay]))
    A = dg.global_matrix().toarray()
    for e in [0, 9, 63]:
        assert abs(A[e, e] - (h * h + dt * h * (abs(ax) + abs(ay)))) < 1e-15
        assert abs(A[e, dg.mesh.neighbor(e, 0)] + dt * h * ax) < 1e-15
        assert abs(A[e, dg.mesh.neighbor(e, 2)] + dt * h * ay) < 1e-15
        assert A[e, dg.mesh.neighbor(e, 1)] == 0.0 and A[e, dg.mesh.neighbor(e, 3)] == 0.0


@pytest.mark.parametrize("dim,n,nel", [(2, 4, (3, 3)), (2, 6, (4, 2)), (3, 3, (2, 3, 2))])
def test_constant_field_annihilates_constants(dim, n, nel):
    vel = synthetic.constant_velocity([0.9, -0.4, 0.3][:dim])
    dg = AdvectionDG(PeriodicMesh(nel), n, 0.3, vel)
    S = dg.global_matrix()
    one = np.ones(dg.ndof)
    Mone = np.concatenate([dg.mass_block(e) @ np.ones(dg.nloc) for e in range(dg.mesh.num_elem)])
    assert np.allclose(S @ one, Mone, atol=1e-14)


@pytest.mark.parametrize("dim,n,nel", [(2, 5, (3, 4)), (3, 3, (2, 2, 3))])
def test_discrete_conservation(dim, n, nel):
    vel = synthetic.fourier_velocity(11, dim)
    dg = AdvectionDG(PeriodicMesh(nel), n, 0.7, vel)
    S = dg.global_matrix()
    x = np.random.default_rng(1).standard_normal(dg.ndof)
    Mx = np.concatenate([dg.mass_block(e) @ x[e * dg.nloc:(e + 1) * dg.nloc]
                         for e in range(dg.mesh.num_elem)])
    # 1^T (S - M) x = dt 1^T A x = 0: volume terms vanish on constants and fluxes cancel
    assert abs(np.sum(S @ x) - np.sum(Mx)) < 1e-12 * np.abs(S @ x).sum()


@pytest.mark.parametrize("dim,n,nel,mu", [(2, 4, (3, 2), None), (2, 3, (2, 2), 5),
                                          (3, 3, (2, 2, 2), None), (3, 2, (2, 1, 2), 4)])
def test_assembly_matches_sum_factorised_matvec(dim, n, nel, mu):
    vel = synthetic.fourier_velocity(5, dim)
    dg = AdvectionDG(PeriodicMesh(nel), n, 0.05, vel, mu=mu)
    x = np.random.default_rng(2).standard_normal(dg.ndof)
    y1 = dg.global_matrix() @ x
    y2 = dg.apply_sumfact(x)
    assert np.linalg.norm(y1 - y2) <= 1e-13 * np.linalg.norm(y1)


def test_periodic_face_points_agree():
    vel = synthetic.fourier_velocity(3, 2)
    dg = AdvectionDG(PeriodicMesh((3, 3)), 4, 0.1, vel)
    for e in range(9):
        for face in range(4):
            nb = dg.mesh.neighbor(e, face)
            opp = face ^ 1
            assert np.array_equal(dg.face_points(e, face), dg.face_points(nb, opp))


@pytest.mark.parametrize("dim,n,nel", [(2, 3, (4, 4)), (2, 6, (5, 5)), (3, 3, (3, 3, 3))])
def test_isolated_blocks_are_mesh_diagonal_blocks(dim, n, nel):
    """Isolated elements at the cell centres of a mesh of the unit cube have the
    mesh operator's diagonal blocks (neighbour couplings dropped)."""
    from oracle.dg import IsolatedElements
    mesh = PeriodicMesh(nel)                       # unit cube, h = 1 / N
    h = mesh.h
    vel = synthetic.fourier_velocity(11, dim)
    dg = AdvectionDG(mesh, n, 0.07, vel)
    centres = np.array([[(c + 0.5) * h for c in mesh.coords(e)] for e in range(mesh.num_elem)])
    iso = IsolatedElements(n, h, centres, 0.07, vel)
    for e in range(mesh.num_elem):
        B = iso.block(e)
        ref = dg.element_block(e)
        assert np.abs(B - ref).max() <= 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("dim,n,nel", [(2, 4, (5, 5)), (3, 3, (3, 3, 3))])
def test_isolated_blocks_unit_elements(dim, n, nel):
    """Unit elements (h = 1) on an N-wide periodic domain: the isolated element with
    width 1 sampling the field over span 1/N at the normalised centre is the mesh's
    diagonal block."""
    from oracle.dg import IsolatedElements
    N = nel[0]
    mesh = PeriodicMesh(nel, 1.0)
    vel = synthetic.fourier_velocity(12, dim)
    dg = AdvectionDG(mesh, n, 0.05, vel)
    centres = np.array([[(c + 0.5) / N for c in mesh.coords(e)] for e in range(mesh.num_elem)])
    iso = IsolatedElements(n, 1.0, centres, 0.05, vel, span=1.0 / N)
    for e in range(mesh.num_elem):
        ref = dg.element_block(e)
        assert np.abs(iso.block(e) - ref).max() <= 1e-13 * np.abs(ref).max()
