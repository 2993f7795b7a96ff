"""Element mass matrices with over-integration and their PCG inversion (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Sec. 3.3, Eq. mass-kron: the mass matrix of element K is
    M_K = (G^T W (x) ... (x) G^T W) J_T (G (x) ... (x) G)
with G the mu x n evaluation matrix of the nodal basis at the mu-point
Gauss-Legendre rule (mu >= n), W its weights and J_T the absolute Jacobian
determinant of the element map at the mu^d quadrature points.  With mu = n the
nodes are the quadrature points (G = I) and M_K is diagonal: the under-integrated
mass matrix the paper uses to precondition an element-wise conjugate-gradient
solve of M_K x = r.

``mass_matrix`` assembles M_K densely (the definition); ``solve`` is the dense
solve; ``pcg`` is the preconditioned conjugate gradient method (Hestenes and
Stiefel, with the preconditioner applied as z = P^-1 r) in its textbook order,
returning the iterate and the number of iterations to ||r|| <= rtol ||b||.

Pinned in tests/test_oracle_mass.py: M_K is symmetric positive definite; for an
affine element M_K = h^d (W (x) W) exactly; for a bilinear element the n-point
rule is already exact (so PCG with the under-integrated preconditioner converges
in one iteration, the paper's observation), and M_K does not change with mu > n;
the PCG iterate equals the dense solve.
"""
from __future__ import annotations

import numpy as np

from .basis import Basis1D


def _kron_all(mats):
    out = mats[0]
    for m in mats[1:]:
        out = np.kron(out, m)
    return out


def quadrature_points(n: int, mu: int, dim: int):
    """Reference points [mu^dim, dim] of the tensor rule, x index fastest, and weights."""
    b = Basis1D(n, mu)
    grids = np.meshgrid(*([b.x] * dim), indexing="ij")
    pts = np.stack(grids, axis=-1)                              # [..x, ..y, (..z), dim]
    pts = np.transpose(pts, tuple(range(dim - 1, -1, -1)) + (dim,)).reshape(-1, dim)
    w = _kron_all([b.w] * dim)                                  # slowest direction left
    return pts, w


def mass_matrix(n: int, mu: int, dim: int, jac_q: np.ndarray) -> np.ndarray:
    """M_K for |J_T| values jac_q at the mu^dim quadrature points (x fastest)."""
    b = Basis1D(n, mu)
    G = _kron_all([b.G] * dim)                                  # [mu^d, n^d]
    _, w = quadrature_points(n, mu, dim)
    return G.T @ ((w * jac_q)[:, None] * G)


def solve(M: np.ndarray, r: np.ndarray) -> np.ndarray:
    return np.linalg.solve(M, r)


def pcg(M: np.ndarray, r: np.ndarray, pdiag: np.ndarray, rtol: float = 1e-12,
        max_iters: int = 200):
    """Preconditioned CG for M x = r from x = 0 with P = diag(pdiag)."""
    x = np.zeros_like(r)
    res = r.copy()
    z = res / pdiag
    p = z.copy()
    rz = res @ z
    nb = np.linalg.norm(r)
    it = 0
    while np.linalg.norm(res) > rtol * nb and it < max_iters:
        Ap = M @ p
        alpha = rz / (p @ Ap)
        x = x + alpha * p
        res = res - alpha * Ap
        it += 1
        z = res / pdiag
        rz_new = res @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, it


def under_integrated_diag(n: int, dim: int, jac_nodes: np.ndarray) -> np.ndarray:
    """Diagonal of the n-point (collocated) mass matrix: w (x) ... (x) w times |J_T| at
    the nodes (x fastest)."""
    b = Basis1D(n)
    return _kron_all([b.w] * dim) * jac_nodes
