"""Pins of the curved-element oracle (oracle/curved.py) on the CPU, in 2D and 3D: the
identity map reproduces the affine operator of oracle/dg.py, the warp's Jacobian against
finite differences, conservation, the area (volume) of the warped domain, the two sides of
a face, and the divergence theorem (free stream) approached with over-integration."""
import numpy as np
import pytest

import synthetic
from oracle.curved import CurvedAdvectionDG
from oracle.dg import AdvectionDG, PeriodicMesh


def _identity(X):
    X = np.asarray(X, dtype=np.float64)
    return X.copy(), np.broadcast_to(np.eye(2), X.shape[:-1] + (2, 2)).copy()


def _warp(L, alpha=0.05):
    return lambda X: synthetic.periodic_warp(X, L, alpha)


@pytest.mark.parametrize("mu", [None, 7])
def test_identity_map_is_the_affine_operator(mu):
    mesh = PeriodicMesh((3, 3), 0.5)
    vel = synthetic.fourier_velocity(1705, 2)
    cur = CurvedAdvectionDG(mesh, 5, 0.05, vel, _identity, mu=mu)
    ref = AdvectionDG(mesh, 5, 0.05, vel, mu).global_matrix()
    S = cur.global_matrix()
    assert abs(S - ref).max() <= 1e-13 * abs(ref).max()


def test_warp_gradient_matches_finite_differences():
    X = np.random.Generator(np.random.PCG64(4)).uniform(0, 2, (20, 2))
    _, G = synthetic.periodic_warp(X, 2.0, 0.07)
    eps = 1e-6
    for j in range(2):
        d = np.zeros(2)
        d[j] = eps
        fd = (synthetic.periodic_warp(X + d, 2.0, 0.07)[0] -
              synthetic.periodic_warp(X - d, 2.0, 0.07)[0]) / (2 * eps)
        assert np.abs(fd - G[:, :, j]).max() <= 1e-8


def test_conservation_and_face_antisymmetry():
    mesh = PeriodicMesh((4, 4), 0.5)
    cur = CurvedAdvectionDG(mesh, 5, 0.05, synthetic.fourier_velocity(1705, 2), _warp(2.0))
    D = (cur.global_matrix() - cur.mass_matrix()).toarray()
    assert np.abs(np.ones(cur.ndof) @ D).max() <= 1e-12 * np.abs(D).max()
    for e in (0, 5, 10):
        for f in range(4):
            nb = mesh.neighbor(e, f)
            a, b = cur.face_an(e, f), cur.face_an(nb, f ^ 1)
            assert np.abs(a + b).max() <= 1e-13 * max(1.0, np.abs(a).max())


def test_warped_area_and_curvature():
    """The masses of all elements add up to the area of the square (the warp preserves
    area; exact up to rounding here, since the periodic part of the determinant sums to
    zero over the cells); a single element's area converges spectrally to a 24-point
    reference; the warped mass is not the affine one."""
    L = 2.0
    mesh = PeriodicMesh((4, 4), L / 4)
    vel = synthetic.fourier_velocity(1705, 2)
    area = {}
    for n in (4, 8, 24):
        cur = CurvedAdvectionDG(mesh, n, 0.05, vel, _warp(L))
        one = np.ones(cur.ndof)
        assert abs(one @ (cur.mass_matrix() @ one) - L * L) <= 1e-12 * L * L
        area[n] = np.ones(cur.nloc) @ cur.mass_block(5) @ np.ones(cur.nloc)
    e4, e8 = abs(area[4] - area[24]), abs(area[8] - area[24])
    assert e8 <= 1e-8 * area[24] and e8 < e4
    cur = CurvedAdvectionDG(mesh, 4, 0.05, vel, _warp(L))
    aff = AdvectionDG(mesh, 4, 0.05, vel)
    assert np.abs(cur.mass_block(5) - aff.mass_block(5)).max() > 1e-3


def test_free_stream_with_over_integration():
    """Constant velocity, u = 1: volume and face terms cancel by the divergence theorem;
    on the warped elements the quadrature error of that identity falls with mu."""
    L = 2.0
    mesh = PeriodicMesh((3, 3), L / 3)
    vel = synthetic.constant_velocity([1.0, 0.5])
    res = []
    for mu in (6, 12, 20):
        cur = CurvedAdvectionDG(mesh, 6, 0.05, vel, _warp(L), mu=mu)
        D = (cur.global_matrix() - cur.mass_matrix())
        res.append(np.linalg.norm(D @ np.ones(cur.ndof)) / abs(D).max())
    assert res[2] <= 1e-9 and res[2] < res[0]


# ---- 3D mapped hexahedra (CurvedAdvectionDG3D) ----------------------------------------
def _identity3(X):
    X = np.asarray(X, dtype=np.float64)
    return X.copy(), np.broadcast_to(np.eye(3), X.shape[:-1] + (3, 3)).copy()


def _warp3(L, alpha=0.03):
    return lambda X: synthetic.periodic_warp3(X, L, alpha)


@pytest.mark.parametrize("mu", [None, 5])
def test_3d_identity_map_is_the_affine_operator(mu):
    from oracle.curved import CurvedAdvectionDG3D
    mesh = PeriodicMesh((2, 3, 2), 0.5)
    vel = synthetic.fourier_velocity(1705, 3)
    S = CurvedAdvectionDG3D(mesh, 3, 0.05, vel, _identity3, mu=mu).global_matrix()
    ref = AdvectionDG(mesh, 3, 0.05, vel, mu).global_matrix()
    assert abs(S - ref).max() <= 1e-13 * abs(ref).max()


def test_3d_warp_gradient_matches_finite_differences():
    X = np.random.Generator(np.random.PCG64(5)).uniform(0, 2, (20, 3))
    _, G = synthetic.periodic_warp3(X, 2.0, 0.04)
    eps = 1e-6
    for j in range(3):
        d = np.zeros(3)
        d[j] = eps
        fd = (synthetic.periodic_warp3(X + d, 2.0, 0.04)[0] -
              synthetic.periodic_warp3(X - d, 2.0, 0.04)[0]) / (2 * eps)
        assert np.abs(fd - G[:, :, j]).max() <= 1e-8


def test_3d_conservation_volume_and_faces():
    """1^T (S - M) = 0 (constant test function: no volume term, face fluxes cancel); the
    mass of the whole warped cube is L^3 (the warp's Jacobian terms sum to zero over a
    period at the element Gauss points); the two sides of every face see opposite scaled
    normal velocities."""
    from oracle.curved import CurvedAdvectionDG3D
    L, N = 2.0, 3
    mesh = PeriodicMesh((N, N, N), L / N)
    dg = CurvedAdvectionDG3D(mesh, 3, 0.1, synthetic.fourier_velocity(1705, 3), _warp3(L))
    D = (dg.global_matrix() - dg.mass_matrix()).toarray()
    assert np.abs(np.ones(dg.ndof) @ D).max() <= 1e-12 * np.abs(D).max()
    vol = sum(dg.volume_geometry(e)[0] @ np.kron(dg.basis.w, np.kron(dg.basis.w, dg.basis.w))
              for e in range(mesh.num_elem))
    assert abs(vol - L ** 3) <= 1e-12 * L ** 3
    for e in range(mesh.num_elem):
        for d in range(3):
            nb = mesh.neighbor(e, 2 * d + 1)
            assert np.abs(dg.face_an(e, 2 * d + 1) + dg.face_an(nb, 2 * d)).max() <= 1e-13


def test_3d_free_stream_with_refined_quadrature():
    """Constant velocity and u = 1: (S - M) 1 = -dt (volume - faces) 1 vanishes by the
    divergence theorem as the quadrature resolves the geometry (spectral decrease)."""
    from oracle.curved import CurvedAdvectionDG3D
    L = 2.0
    mesh = PeriodicMesh((3, 3, 3), L / 3)
    vel = synthetic.constant_velocity([1.0, -0.5, 0.25])
    res = []
    for mu in (3, 5, 8):
        dg = CurvedAdvectionDG3D(mesh, 3, 1.0, vel, _warp3(L), mu=mu)
        D = dg.global_matrix() - dg.mass_matrix()
        res.append(np.linalg.norm(D @ np.ones(dg.ndof)) / abs(D).max())
    # measured 3.8e-3, 1.6e-7, 1.2e-14
    assert res[0] > 1e-4 and res[1] < 1e-3 * res[0] and res[2] <= 1e-12, res


def test_3d_warp_is_periodic_and_orientation_preserving():
    """Phi(X + L e_d) = Phi(X) + L e_d with the same gradient (the warped elements conform
    across the periodic boundary), and det grad Phi > 0 everywhere."""
    L = 2.0
    X = np.random.Generator(np.random.PCG64(9)).uniform(0, L, (50, 3))
    x0, G0 = synthetic.periodic_warp3(X, L, 0.03)
    for d in range(3):
        sh = np.zeros(3)
        sh[d] = L
        x1, G1 = synthetic.periodic_warp3(X + sh, L, 0.03)
        assert np.abs(x1 - x0 - sh).max() <= 1e-13 and np.abs(G1 - G0).max() <= 1e-12
    g = np.linspace(0, L, 17)
    P = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    assert np.linalg.det(synthetic.periodic_warp3(P, L, 0.03)[1]).min() > 0.3
