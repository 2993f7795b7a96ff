"""GPU: element-wise PCG inversion of the exact (over-integrated) mass matrix with the
under-integrated preconditioner (Sec. 3.3) against the oracle's dense solve and PCG."""
import numpy as np
import pytest

import synthetic
from oracle import mass
from paper_1704_04549_gb300 import Context, mesh
from tests.gpu_util import DEV, rel, to_dev, to_host

pytestmark = pytest.mark.gpu


def _ctx(dim, n, E, nrhs=1):
    nb = mesh.isolated_nbr(E, dim)
    z = np.zeros(dim * E * n ** dim)
    zf = np.zeros(E * 2 * dim * n ** (dim - 1))
    return Context.from_arrays(dim, n, 1.0, 0.05, nb, z, zf, nrhs=nrhs, device=DEV)


def _jacobians(maps, n, mu, dim):
    pts, _ = mass.quadrature_points(n, mu, dim)
    nodes, _ = mass.quadrature_points(n, n, dim)
    E = maps.num_elem
    jq = np.stack([maps.jacobian(e, pts) for e in range(E)])
    jn = np.stack([maps.jacobian(e, nodes) for e in range(E)])
    return jq, jn


@pytest.mark.parametrize("dim,n,mu,kind", [(2, 4, 6, "curved"), (2, 16, 20, "curved"),
                                           (2, 31, 34, "curved"), (2, 7, 10, "bilinear"),
                                           (3, 4, 6, "curved"), (3, 8, 11, "curved"),
                                           (2, 5, 5, "affine")])
def test_mass_solve_matches_oracle(dim, n, mu, kind):
    """Every element block: x equals the oracle's dense solve (rtol 1e-12 PCG), and the
    iteration count equals the oracle PCG's (+-1); bilinear and affine elements take one
    iteration (the n-point rule is exact there)."""
    E, R = 6, 2
    maps = synthetic.element_maps(21, E, dim, kind, h=0.25, eps=0.1)
    jq, jn = _jacobians(maps, n, mu, dim)
    ctx = _ctx(dim, n, E, R)
    nl = n ** dim
    b = synthetic.rhs(31, E * R * nl)
    x, its, st = ctx.tpp_mass_solve(mu, jq, jn, to_dev(b), rtol=1e-12)
    X, its = to_host(x).reshape(E, R, nl), to_host(its).reshape(E, R)
    B = b.reshape(E, R, nl)
    for e in range(E):
        M = mass.mass_matrix(n, mu, dim, jq[e])
        P = mass.under_integrated_diag(n, dim, jn[e])
        for r in range(R):
            ref = mass.solve(M, B[e, r])
            assert rel(X[e, r], ref) <= 1e-11 * np.linalg.cond(M), (e, r)
            _, it_ref = mass.pcg(M, B[e, r], P, rtol=1e-12)
            assert abs(int(its[e, r]) - it_ref) <= 1, (e, r, its[e, r], it_ref)
            if kind in ("bilinear", "affine") and dim == 2:
                assert its[e, r] == 1
    print(f"mass PCG dim={dim} n={n} mu={mu} {kind}: iterations {sorted(set(its.ravel()))}")


def test_mass_solve_limits():
    ctx = _ctx(2, 4, 2)
    maps = synthetic.element_maps(2, 2, 2, "curved")
    jq, jn = _jacobians(maps, 4, 6, 2)
    b = to_dev(synthetic.rhs(3, 2 * 16))
    with pytest.raises(Exception):
        ctx.tpp_mass_solve(3, jq[:, :9], jn, b)              # mu < n
    x, its, st = ctx.tpp_mass_solve(6, jq, jn, b, rtol=1e-15, max_iters=2, check=False)
    assert st == 4 and int(to_host(its).max()) == 2          # iteration limit reported
