"""Restarted, right-preconditioned GMRES and flexible GMRES (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper solves each linear system with "preconditioned, restarted GMRES"
(Sec. 5, opening paragraph) without fixing the side, the restart length or
the orthogonalisation.  Readings used here: right preconditioning (so the
Arnoldi residual estimate is the true unpreconditioned residual in exact
arithmetic), x0 = 0, restart m = 30, modified Gram-Schmidt Arnoldi, Givens
rotations for the least-squares problem (Saad, Alg. 6.9 / 9.5).  A cycle
ends when the Arnoldi estimate |g_{j+1}| <= rtol ||b|| or after m steps; the
true residual ||b - A x|| / ||b|| is then computed and the solve stops when
it is <= rtol.  The flexible variant stores Z = [P^-1 v_1, ...] and forms
x = x0 + Z y, which stays exact when P^-1 is applied in reduced precision.

Pinned in tests/test_oracle_gmres.py: one iteration with the exact inverse
as preconditioner on a block-diagonal system, agreement with scipy's sparse
direct solve, and the iteration count matching an unrestarted run's
residual history.
"""
from __future__ import annotations

import numpy as np


def gmres(A, b: np.ndarray, M=None, restart: int = 30, rtol: float = 1e-8,
          max_iters: int = 3000, flexible: bool = False):
    """Solve A x = b.  A and M are callables (M = P^-1, right preconditioner).

    Returns (x, info) with info = dict(iters, true_rel_res, history, converged)."""
    M = (lambda v: v) if M is None else M
    nb = np.linalg.norm(b)
    x = np.zeros_like(b)
    info = dict(iters=0, history=[], converged=False, true_rel_res=1.0)
    if nb == 0.0:
        info.update(converged=True, true_rel_res=0.0)
        return x, info
    r = b - A(x)
    beta = np.linalg.norm(r)
    total = 0
    while total < max_iters:
        m = restart
        V = np.zeros((b.shape[0], m + 1))
        Z = np.zeros((b.shape[0], m)) if flexible else None
        H = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[:, 0] = r / beta
        k = 0
        for j in range(m):
            z = M(V[:, j])
            if flexible:
                Z[:, j] = z
            w = A(z)
            for i in range(j + 1):                      # modified Gram-Schmidt
                H[i, j] = np.dot(w, V[:, i])
                w = w - H[i, j] * V[:, i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] > 0.0:
                V[:, j + 1] = w / H[j + 1, j]
            for i in range(j):                          # previous rotations
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            rho = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / rho, H[j + 1, j] / rho
            H[j, j], H[j + 1, j] = rho, 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            total += 1
            k = j + 1
            info["history"].append(abs(g[j + 1]) / nb)
            if abs(g[j + 1]) <= rtol * nb or total >= max_iters:
                break
        y = np.linalg.solve(np.triu(H[:k, :k]), g[:k])
        if flexible:
            x = x + Z[:, :k] @ y
        else:
            x = x + M(V[:, :k] @ y)
        r = b - A(x)
        beta = np.linalg.norm(r)
        info["true_rel_res"] = beta / nb
        if beta <= rtol * nb:
            info["converged"] = True
            break
    info["iters"] = total
    return x, info
