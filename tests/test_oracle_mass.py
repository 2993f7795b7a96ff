"""Pins of the mass-matrix oracle (Sec. 3.3): symmetry and definiteness, the affine
closed form, exactness of the n-point rule on bilinear elements (and hence one PCG
iteration with the under-integrated preconditioner), and PCG = dense solve."""
import numpy as np
import pytest

import synthetic
from oracle import mass
from oracle.basis import Basis1D


def _jac(maps, e, n, mu, dim):
    pts, _ = mass.quadrature_points(n, mu, dim)
    nodes, _ = mass.quadrature_points(n, n, dim)
    return maps.jacobian(e, pts), maps.jacobian(e, nodes)


@pytest.mark.parametrize("dim,n", [(2, 3), (2, 6), (3, 3)])
def test_affine_mass_is_the_weight_diagonal(dim, n):
    maps = synthetic.element_maps(1, 1, dim, "affine", h=0.5)
    for mu in (n, n + 2):
        jq, _ = _jac(maps, 0, n, mu, dim)
        M = mass.mass_matrix(n, mu, dim, jq)
        w = Basis1D(n).w
        ref = np.diag(mass._kron_all([w] * dim)) * 0.5 ** dim
        assert np.abs(M - ref).max() <= 1e-14


@pytest.mark.parametrize("kind", ["bilinear", "curved"])
def test_mass_is_spd_and_pcg_solves_it(kind):
    dim, n, mu = 2, 5, 8
    maps = synthetic.element_maps(2, 3, dim, kind, eps=0.1)
    for e in range(3):
        jq, jn = _jac(maps, e, n, mu, dim)
        M = mass.mass_matrix(n, mu, dim, jq)
        assert np.abs(M - M.T).max() <= 1e-15 * np.abs(M).max()
        assert np.linalg.eigvalsh(M).min() > 0
        r = synthetic.rhs(5 + e, n ** dim)
        x, it = mass.pcg(M, r, mass.under_integrated_diag(n, dim, jn))
        assert np.linalg.norm(x - mass.solve(M, r)) <= 1e-11 * np.linalg.norm(x)


@pytest.mark.parametrize("n", [2, 4, 7])
def test_bilinear_elements_need_one_iteration(n):
    """A bilinear map has a linear Jacobian determinant, so the n-point Gauss rule
    integrates u v |J| exactly: the under-integrated mass matrix is the exact one and
    PCG converges in one iteration (Sec. 3.3); over-integration changes nothing."""
    dim = 2
    maps = synthetic.element_maps(3, 2, dim, "bilinear", eps=0.15)
    for e in range(2):
        jq, jn = _jac(maps, e, n, n + 3, dim)
        M = mass.mass_matrix(n, n + 3, dim, jq)
        Mn = mass.mass_matrix(n, n, dim, jn)
        assert np.abs(M - Mn).max() <= 1e-14 * np.abs(M).max()
        r = synthetic.rhs(9, n ** dim)
        _, it = mass.pcg(M, r, mass.under_integrated_diag(n, dim, jn))
        assert it == 1


def test_curved_elements_iterations_do_not_grow_with_p():
    """Curved (non-polynomial) maps: the n-point rule is no longer exact, PCG takes a
    few iterations, and their number does not grow with p (Sec. 3.3)."""
    dim = 2
    maps = synthetic.element_maps(4, 1, dim, "curved", eps=0.1)
    its = []
    for n in (4, 8, 12, 16):
        jq, jn = _jac(maps, 0, n, n + 4, dim)
        M = mass.mass_matrix(n, n + 4, dim, jq)
        r = synthetic.rhs(10, n ** dim)
        _, it = mass.pcg(M, r, mass.under_integrated_diag(n, dim, jn), rtol=1e-10)
        its.append(it)
    assert max(its) <= 12 and its[-1] <= its[0] + 3, its
