"""Time integration of the semi-discrete DG system (oracle; test infrastructure).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The semi-discrete equations read M u' = J u (Sec. 3.3, Eq. mass-u-r with r = J u
for linear advection; J = -A, so S = M + dt A = M - dt J).  Three integrators,
written from their published definitions with dense / sparse direct solves:

* backward Euler: (M - dt J) u^{n+1} = M u^n  (the "one backward Euler step" of
  Sec. 5.3-5.6);
* the three-stage, third-order, L-stable DIRK method of Alexander (1977), used in
  Sec. 5.2: stage values U_i solve (M - gamma dt J) U_i = M (u^n + dt sum_{j<i}
  a_ij k_j), k_i = (U_i - u^n - dt sum_{j<i} a_ij k_j) / (gamma dt) = M^-1 J U_i,
  and u^{n+1} = u^n + dt sum_i b_i k_i (= U_3: the method is stiffly accurate);
* the classical fourth-order explicit Runge-Kutta method (the explicit
  comparison of Sec. 5.2), k_i = M^-1 J (u^n + dt c_i k_{i-1}).

``exact`` is the semi-discrete solution exp(t M^-1 J) u^0 (scipy's expm).

Pinned in tests/test_oracle_timestep.py: the DIRK coefficients satisfy the order
conditions up to order 3 and its stability function vanishes at infinity; each
method's error against ``exact`` falls with the order its definition promises
(1, 3, 4) when dt is halved; all conserve 1^T M u on a periodic mesh.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def alexander_dirk3():
    """(A, b, c) of Alexander's three-stage, third-order, L-stable SDIRK method:
    gamma the root in (1/6, 1/2) of gamma^3 - 3 gamma^2 + 3/2 gamma - 1/6 = 0,
    tau = (1 + gamma) / 2, b_1 = -(6 gamma^2 - 16 gamma + 1) / 4,
    b_2 = (6 gamma^2 - 20 gamma + 5) / 4, A = [[gamma], [tau - gamma, gamma],
    [b_1, b_2, gamma]], b = last row of A, c = (gamma, tau, 1)."""
    roots = np.roots([1.0, -3.0, 1.5, -1.0 / 6.0])
    g = float(next(r.real for r in roots if abs(r.imag) < 1e-12 and 1 / 6 < r.real < 0.5))
    tau = 0.5 * (1.0 + g)
    b1 = -(6 * g * g - 16 * g + 1) / 4
    b2 = (6 * g * g - 20 * g + 5) / 4
    A = np.array([[g, 0.0, 0.0], [tau - g, g, 0.0], [b1, b2, g]])
    return A, A[2].copy(), np.array([g, tau, 1.0])


def _mass_vector(dg) -> np.ndarray:
    """Diagonal of the collocated mass matrix h^d (w (x) ... (x) w) of every element."""
    w = dg.basis.w
    m = w
    for _ in range(dg.dim - 1):
        m = np.kron(w, m)
    return np.tile(dg.mesh.h ** dg.dim * m, dg.mesh.num_elem)


def spatial_operator(dg):
    """(m, J): the mass diagonal and the sparse J = (M - S) / dt of the oracle's
    assembled S = M - dt J (dg.dt > 0)."""
    m = _mass_vector(dg)
    S = dg.global_matrix()
    J = (sp.diags(m) - S) / dg.dt
    return m, sp.csr_matrix(J)


def backward_euler(m, J, u0, dt, steps):
    lu = spla.splu(sp.csc_matrix(sp.diags(m) - dt * J))
    u = np.array(u0, dtype=np.float64)
    for _ in range(steps):
        u = lu.solve(m * u)
    return u


def dirk3(m, J, u0, dt, steps):
    A, b, _ = alexander_dirk3()
    g = A[0, 0]
    lu = spla.splu(sp.csc_matrix(sp.diags(m) - g * dt * J))
    u = np.array(u0, dtype=np.float64)
    for _ in range(steps):
        k = []
        for i in range(3):
            uhat = u + dt * sum(A[i, j] * k[j] for j in range(i))
            U = lu.solve(m * uhat)
            k.append((U - uhat) / (g * dt))
        u = u + dt * sum(b[i] * k[i] for i in range(3))
    return u


def rk4(m, J, u0, dt, steps):
    f = lambda v: (J @ v) / m          # noqa: E731  (M is diagonal)
    u = np.array(u0, dtype=np.float64)
    for _ in range(steps):
        k1 = f(u)
        k2 = f(u + 0.5 * dt * k1)
        k3 = f(u + 0.5 * dt * k2)
        k4 = f(u + dt * k3)
        u = u + dt / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
    return u


def exact(m, J, u0, t):
    """exp(t M^-1 J) u0 (dense; small problems only)."""
    L = (J.toarray() if sp.issparse(J) else J) / m[:, None]
    return sla.expm(t * L) @ u0
