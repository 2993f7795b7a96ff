"""Pins of the linearised system oracle (oracle/systems.py) on the CPU: the Euler
Jacobians against finite differences of the flux of Eq. euler-flux and against the
known characteristic speeds, the one-component reduction to the upwind advection
operator, discrete conservation of every component, and the assembled Jacobian
against a finite difference of the nonlinear DG residual."""
import numpy as np
import pytest

import synthetic
from oracle.dg import AdvectionDG, PeriodicMesh
from oracle.systems import (NORMALS, EulerFlux, LinearAdvectionFlux, LinearizedSystemDG,
                            euler_flux, euler_jacobians, vortex_system)

GAMMA = 1.4


def _states(seed, m):
    rng = np.random.Generator(np.random.PCG64(seed))
    rho = rng.uniform(0.5, 2.0, m)
    u, v = rng.uniform(-1, 1, m), rng.uniform(-1, 1, m)
    p = rng.uniform(0.5, 3.0, m)
    E = p / ((GAMMA - 1) * rho) + 0.5 * (u * u + v * v)
    return np.stack([rho, rho * u, rho * v, rho * E], -1)


def test_euler_jacobians_match_finite_differences():
    U = _states(1, 20)
    Ax, Ay = euler_jacobians(U, GAMMA)
    eps = 1e-6
    for k in range(4):
        d = np.zeros(4)
        d[k] = eps
        F1p, F2p = euler_flux(U + d, GAMMA)
        F1m, F2m = euler_flux(U - d, GAMMA)
        fd1, fd2 = (F1p - F1m) / (2 * eps), (F2p - F2m) / (2 * eps)
        assert np.abs(fd1 - Ax[:, :, k]).max() <= 1e-7 * max(1, np.abs(Ax).max())
        assert np.abs(fd2 - Ay[:, :, k]).max() <= 1e-7 * max(1, np.abs(Ay).max())


def test_normal_jacobian_eigenvalues_are_the_characteristic_speeds():
    U = _states(2, 10)
    Ax, Ay = euler_jacobians(U, GAMMA)
    rho, u, v = U[:, 0], U[:, 1] / U[:, 0], U[:, 2] / U[:, 0]
    p = (GAMMA - 1) * (U[:, 3] - 0.5 * rho * (u * u + v * v))
    c = np.sqrt(GAMMA * p / rho)
    for nx, ny in [(1.0, 0.0), (0.0, -1.0), (0.6, 0.8)]:
        An = nx * Ax + ny * Ay
        vn = u * nx + v * ny
        for q in range(U.shape[0]):
            ev = np.sort(np.linalg.eigvals(An[q]).real)
            ref = np.sort([vn[q] - c[q], vn[q], vn[q], vn[q] + c[q]])
            assert np.abs(ev - ref).max() <= 1e-10 * (abs(vn[q]) + c[q])


@pytest.mark.parametrize("a", [(1.0, 0.5), (-0.7, 0.3)])
def test_one_component_system_is_upwind_advection(a):
    """LLF with lam = |a.n| is the upwind flux: the system operator of F(u) = a u equals
    the scalar advection operator of oracle/dg.py."""
    mesh = PeriodicMesh((3, 4), 0.25)
    n, dt = 4, 0.1
    sysdg = LinearizedSystemDG(mesh, n, dt, LinearAdvectionFlux(a),
                               np.zeros((mesh.num_elem, 1, n * n)))
    ref = AdvectionDG(mesh, n, dt, synthetic.constant_velocity(list(a))).global_matrix()
    S = sysdg.global_matrix()
    assert abs(S - ref).max() <= 1e-13 * abs(ref).max()


def test_every_component_is_conserved():
    """1_c^T (S - M) = 0: volume terms of a constant test function vanish and the LLF
    face fluxes of the two sides of a face cancel."""
    sysdg = vortex_system((4, 3), 2.5, 3, 0.1, synthetic.euler_vortex_state)
    D = (sysdg.global_matrix() - sysdg.mass_matrix()).toarray()
    for c in range(4):
        one = np.zeros(sysdg.ndof)
        for e in range(sysdg.mesh.num_elem):
            one[e * sysdg.bs + c * sysdg.nloc:e * sysdg.bs + (c + 1) * sysdg.nloc] = 1.0
        assert np.abs(one @ D).max() <= 1e-12 * np.abs(D).max()


def test_jacobian_matches_the_nonlinear_residual():
    sysdg = vortex_system((4, 4), 2.5, 3, 0.1, synthetic.euler_vortex_state)
    lam = [[sysdg.face_data(e, f)[2] for f in range(4)] for e in range(sysdg.mesh.num_elem)]
    D = sysdg.global_matrix() - sysdg.mass_matrix()
    x = synthetic.rhs(5, sysdg.ndof) * 0.01 * np.abs(sysdg.U0.reshape(-1)).max()
    eps = 1e-4
    U0 = sysdg.U0.reshape(-1)
    fd = (sysdg.residual(U0 + eps * x, lam) - sysdg.residual(U0 - eps * x, lam)) / (2 * eps)
    ref = D @ x
    assert np.linalg.norm(fd - ref) <= 1e-6 * np.linalg.norm(ref)


def test_vortex_state_is_isentropic_and_faces_are_outflow_dominated():
    """p / rho^gamma is constant for the vortex (Sec. 5.3), and with the LLF speed the
    small blocks' own-face coefficients 1/2 (A_n[c, c] + lam) are non-negative."""
    X = np.random.Generator(np.random.PCG64(3)).uniform(0, 15, (200, 2))
    U = synthetic.euler_vortex_state(X)
    rho = U[:, 0]
    u, v = U[:, 1] / rho, U[:, 2] / rho
    p = (GAMMA - 1) * (U[:, 3] - 0.5 * rho * (u * u + v * v))
    s = p / rho ** GAMMA
    assert np.abs(s / s[0] - 1).max() <= 1e-12
    sysdg = vortex_system((4, 4), 2.5, 4, 0.1, synthetic.euler_vortex_state)
    for e in range(sysdg.mesh.num_elem):
        for f in range(4):
            own, _, _ = sysdg.face_data(e, f)
            assert np.diagonal(own, axis1=1, axis2=2).min() >= 0.0


# ---- 3D (five components) ----------------------------------------------------------
def _states3d(seed, m):
    rng = np.random.Generator(np.random.PCG64(seed))
    rho = rng.uniform(0.5, 2.0, m)
    V = rng.uniform(-1, 1, (m, 3))
    p = rng.uniform(0.5, 3.0, m)
    E = p / ((GAMMA - 1) * rho) + 0.5 * np.sum(V * V, -1)
    return np.concatenate([rho[:, None], rho[:, None] * V, (rho * E)[:, None]], -1)


def test_euler3d_jacobians_and_speeds():
    from oracle.systems import euler3d_flux, euler3d_jacobians
    U = _states3d(6, 15)
    A = euler3d_jacobians(U, GAMMA)
    eps = 1e-6
    for k in range(5):
        d = np.zeros(5)
        d[k] = eps
        Fp, Fm = euler3d_flux(U + d, GAMMA), euler3d_flux(U - d, GAMMA)
        for dd in range(3):
            fd = (Fp[dd] - Fm[dd]) / (2 * eps)
            assert np.abs(fd - A[dd][:, :, k]).max() <= 1e-7 * max(1, np.abs(A[dd]).max())
    rho = U[:, 0]
    V = U[:, 1:4] / rho[:, None]
    p = (GAMMA - 1) * (U[:, 4] - 0.5 * rho * np.sum(V * V, -1))
    c = np.sqrt(GAMMA * p / rho)
    nv = np.array([0.48, 0.6, 0.64])
    for q in range(U.shape[0]):
        An = sum(nv[d] * A[d][q] for d in range(3))
        vn = V[q] @ nv
        ev = np.sort(np.linalg.eigvals(An).real)
        ref = np.sort([vn - c[q], vn, vn, vn, vn + c[q]])
        assert np.abs(ev - ref).max() <= 1e-9 * (abs(vn) + c[q])


def test_one_component_system_is_upwind_advection_3d():
    mesh = PeriodicMesh((2, 3, 2), 0.5)
    a = (1.0, -0.5, 0.3)
    n = 3
    sysdg = LinearizedSystemDG(mesh, n, 0.1, LinearAdvectionFlux(a),
                               np.zeros((mesh.num_elem, 1, n ** 3)))
    ref = AdvectionDG(mesh, n, 0.1, synthetic.constant_velocity(list(a))).global_matrix()
    assert abs(sysdg.global_matrix() - ref).max() <= 1e-13 * abs(ref).max()


def test_3d_conservation_and_residual():
    L = 2.0
    sysdg = vortex_system((2, 2, 2), L / 2, 3, 0.05,
                          lambda X: synthetic.euler3d_wave_state(X, L))
    D = sysdg.global_matrix() - sysdg.mass_matrix()
    Dd = D.toarray()
    for c in range(5):
        one = np.zeros(sysdg.ndof)
        for e in range(sysdg.mesh.num_elem):
            one[e * sysdg.bs + c * sysdg.nloc:e * sysdg.bs + (c + 1) * sysdg.nloc] = 1.0
        assert np.abs(one @ Dd).max() <= 1e-12 * np.abs(Dd).max()
    lam = [[sysdg.face_data(e, f)[2] for f in range(6)] for e in range(sysdg.mesh.num_elem)]
    x = synthetic.rhs(8, sysdg.ndof) * 0.01
    eps = 1e-4
    U0 = sysdg.U0.reshape(-1)
    fd = (sysdg.residual(U0 + eps * x, lam) - sysdg.residual(U0 - eps * x, lam)) / (2 * eps)
    assert np.linalg.norm(fd - D @ x) <= 1e-6 * np.linalg.norm(D @ x)


# ---- full-block KSVD (Sec. 5.3: A_k of size n_c (p+1)) ---------------------------
def test_full_block_ksvd_reduces_to_the_scalar_ksvd():
    """One component: the full block is the scalar block and its KSVD the scalar one."""
    from oracle.ksvd import kron_sum, ksvd_2d
    mesh = PeriodicMesh((3, 2), 0.5)
    n = 4
    sysdg = LinearizedSystemDG(mesh, n, 0.1, LinearAdvectionFlux((1.0, -0.4)),
                               np.zeros((mesh.num_elem, 1, n * n)))
    for e in (0, 4):
        s, As, Bs = sysdg.full_block_ksvd(e)
        s_ref, Ar, Br = ksvd_2d(sysdg.element_block(e), n)
        assert np.abs(s[:2] - s_ref[:2]).max() <= 1e-13 * s_ref[0]
        P, Pr = kron_sum(As, Bs), kron_sum(Ar, Br)
        assert np.abs(P - Pr).max() <= 1e-12 * np.abs(Pr).max()


def test_full_block_ksvd_exact_for_the_mass():
    """dt = 0: S_e = I_(n_c) (x) h^2 diag(w) (x) diag(w) = (I (x) h^2 diag(w)) (x) diag(w),
    rank 1 in the (component, y) x (x) split: the approximation is exact and
    sigma_1 = h^2 ||w||^2 sqrt(n_c)."""
    from oracle.ksvd import kron_sum
    n, h = 5, 2.5
    sysdg = vortex_system((3, 3), h, n, 0.0, synthetic.euler_vortex_state)
    s, As, Bs = sysdg.full_block_ksvd(4)
    S = sysdg.element_block(4)
    assert np.abs(kron_sum(As, Bs) - S).max() <= 1e-13 * np.abs(S).max()
    w = 0.5 * np.polynomial.legendre.leggauss(n)[1]
    assert abs(s[0] - h * h * np.sum(w * w) * 2.0) <= 1e-13 * s[0]
    assert s[1] <= 1e-13 * s[0]


def test_full_block_nested_ksvd_3d_reduces_to_the_scalar_one():
    from oracle.ksvd import ksvd_3d_nested
    mesh = PeriodicMesh((2, 2, 2), 0.5)
    n = 3
    sysdg = LinearizedSystemDG(mesh, n, 0.1, LinearAdvectionFlux((1.0, -0.5, 0.3)),
                               np.zeros((mesh.num_elem, 1, n ** 3)))
    for e in (0, 6):
        out = sysdg.full_block_ksvd_3d(e)
        ref = ksvd_3d_nested(sysdg.element_block(e), n)
        assert np.abs(out["P"] - ref["P"]).max() <= 1e-12 * np.abs(ref["P"]).max()


def test_full_block_nested_ksvd_3d_exact_for_the_mass():
    L = 2.0
    n = 3
    sysdg = vortex_system((2, 2, 2), L / 2, n, 0.0, lambda X: synthetic.euler3d_wave_state(X, L))
    out = sysdg.full_block_ksvd_3d(3)
    S = sysdg.element_block(3)
    assert np.abs(out["P"] - S).max() <= 1e-13 * np.abs(S).max()
