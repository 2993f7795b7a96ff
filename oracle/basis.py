"""1D nodal basis and tensor-product quadrature (oracle; test infrastructure).

Follows Sec. 3.1 (tensor-product nodal basis, Eq. tensor-basis) and Sec. 3.2
(evaluation matrix G_{alpha j} = phi_j(x_alpha), differentiation matrix
D_{alpha j} = phi_j'(x_alpha), weight matrix W = diag(w)).

Reading: the nodes B are the n Gauss-Legendre points of [0, 1] and the
quadrature is the same rule (mu = n, so G = I up to rounding); ``mu`` may be
given larger for over-integration.

Pinned in tests/test_oracle_basis.py by closed-form Gauss-Legendre rules,
exact integration of monomials of degree <= 2n-1 and exact differentiation
and endpoint evaluation of random polynomials of degree <= n-1.
"""
from __future__ import annotations

import numpy as np


def gauss_legendre_01(n: int):
    """Gauss-Legendre points and weights mapped from [-1, 1] to [0, 1]."""
    xi, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (xi + 1.0), 0.5 * w


def lagrange_values(nodes: np.ndarray, x) -> np.ndarray:
    """V[a, j] = phi_j(x_a): the degree n-1 Lagrange polynomial of node j.

    Direct product formula phi_j(x) = prod_{m != j} (x - b_m) / (b_j - b_m).
    """
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = nodes.shape[0]
    V = np.ones((x.shape[0], n))
    for j in range(n):
        for m in range(n):
            if m != j:
                V[:, j] *= (x - nodes[m]) / (nodes[j] - nodes[m])
    return V


def lagrange_derivatives(nodes: np.ndarray, x) -> np.ndarray:
    """Dv[a, j] = phi_j'(x_a) by the product rule applied to the formula above:

    phi_j'(x) = sum_{m != j} 1/(b_j - b_m) prod_{k != j, m} (x - b_k)/(b_j - b_k).
    """
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = nodes.shape[0]
    Dv = np.zeros((x.shape[0], n))
    for j in range(n):
        for m in range(n):
            if m == j:
                continue
            term = np.full(x.shape[0], 1.0 / (nodes[j] - nodes[m]))
            for k in range(n):
                if k != j and k != m:
                    term *= (x - nodes[k]) / (nodes[j] - nodes[k])
            Dv[:, j] += term
    return Dv


class Basis1D:
    """Nodal basis of P^p([0,1]) on n = p + 1 Gauss-Legendre nodes.

    Attributes (Sec. 3.2 notation):
      nodes, w   : quadrature points x_alpha and weights (mu points)
      G          : mu x n evaluation matrix, G[a, j] = phi_j(x_a)
      D          : mu x n differentiation matrix, D[a, j] = phi_j'(x_a)
      l0, l1     : phi_j(0), phi_j(1) (face evaluation vectors)
    """

    def __init__(self, n: int, mu: int | None = None):
        self.n = n
        self.mu = n if mu is None else mu
        self.b, _ = gauss_legendre_01(n)          # DG nodes B
        self.x, self.w = gauss_legendre_01(self.mu)  # quadrature
        self.G = lagrange_values(self.b, self.x)
        self.D = lagrange_derivatives(self.b, self.x)
        self.l0 = lagrange_values(self.b, 0.0)[0]
        self.l1 = lagrange_values(self.b, 1.0)[0]
        self.W = np.diag(self.w)
