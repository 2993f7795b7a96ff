"""Preconditioner application (oracle; test infrastructure).

* ``apply_dense``: x = P^-1 b by LU of the assembled matrix (the definition).
* ``factor_2d`` / ``apply_2d``: the paper's route, Alg. 2d-form / 2d-apply
  (Sec. 4.2): multiply P x = b on the left by A_2^-1 (x) B_1^-1, take real Schur
  forms C_1 = A_2^-1 A_1 = Q_1 T_1 Q_1^T and C_2 = B_1^-1 B_2 = Q_2 T_2 Q_2^T
  (Eq. quad-triang) and solve the Sylvester system (T_1 (x) I + I (x) T_2).
  With X the n x n matrix whose column-major vec is x, (A (x) B) vec(X) =
  vec(B X A^T), so the system reads T_2 Y + Y T_1^T = C.
* ``factor_3d`` / ``apply_3d``: Alg. 3d-form / 3d-apply (Sec. 4.3), with
  left multiplication by A_1^-1 (x) B_2^-1 (x) C_1^-1 and Schur forms of
  B_2^-1 B_1 and C_1^-1 C_2; one Sylvester solve per z-slice.
* ``BlockPrecond``: applies per-element inverses to a global vector; exact
  block Jacobi uses LU of the exact diagonal blocks (the comparator of Sec. 5).

Pinned in tests/test_oracle_precond.py: the Schur/Sylvester routes agree with
dense LU of the assembled P, the dt -> 0 limit reduces P to the (rank-one)
mass matrix, and tiny cases are checked against brute-force inverses.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def apply_dense(P: np.ndarray, b: np.ndarray) -> np.ndarray:
    return sla.lu_solve(sla.lu_factor(P), b)


def factor_2d(A1, B1, A2, B2):
    """Alg. 2d-form after the KSVD: LU of A_2 and B_1, real Schur of C_1, C_2."""
    luA2, luB1 = sla.lu_factor(A2), sla.lu_factor(B1)
    C1 = sla.lu_solve(luA2, A1)
    C2 = sla.lu_solve(luB1, B2)
    T1, Q1 = sla.schur(C1, output="real")
    T2, Q2 = sla.schur(C2, output="real")
    return dict(luA2=luA2, luB1=luB1, Q1=Q1, T1=T1, Q2=Q2, T2=T2)


def apply_2d(f, b: np.ndarray) -> np.ndarray:
    """Alg. 2d-apply on one element vector b (length n^2, x fastest)."""
    n = f["Q1"].shape[0]
    Bm = b.reshape((n, n), order="F")                 # Bm[i, j]: i = x, j = y
    # b~ = (A_2^-1 (x) B_1^-1) b  <=>  B_1^-1 Bm A_2^-T
    Bt = sla.lu_solve(f["luB1"], Bm)
    Bt = sla.lu_solve(f["luA2"], Bt.T).T
    # (Q_1^T (x) Q_2^T) b~
    C = f["Q2"].T @ Bt @ f["Q1"]
    # (T_1 (x) I + I (x) T_2) y = c  <=>  T_2 Y + Y T_1^T = C
    Y = sla.solve_sylvester(f["T2"], f["T1"].T, C)
    X = f["Q2"] @ Y @ f["Q1"].T
    return X.reshape(-1, order="F")


def factor_3d(A1, B1, C1, B2, C2):
    """Alg. 3d-form after the nested KSVD: LU of A_1, B_2, C_1; Schur of
    B_2^-1 B_1 and C_1^-1 C_2."""
    luA1, luB2, luC1 = sla.lu_factor(A1), sla.lu_factor(B2), sla.lu_factor(C1)
    T1, Q1 = sla.schur(sla.lu_solve(luB2, B1), output="real")
    T2, Q2 = sla.schur(sla.lu_solve(luC1, C2), output="real")
    return dict(luA1=luA1, luB2=luB2, luC1=luC1, Q1=Q1, T1=T1, Q2=Q2, T2=T2)


def apply_3d(f, b: np.ndarray) -> np.ndarray:
    """Alg. 3d-apply on one element vector b (length n^3, x fastest)."""
    n = f["Q1"].shape[0]
    Bt = b.reshape((n, n, n), order="F")              # Bt[i, j, k]: x, y, z
    # (A_1^-1 (x) B_2^-1 (x) C_1^-1) b: one 1D solve along each direction
    Bt = sla.lu_solve(f["luC1"], Bt.reshape(n, n * n, order="F")).reshape((n, n, n), order="F")
    Bt = np.stack([sla.lu_solve(f["luB2"], Bt[:, :, k].T).T for k in range(n)], axis=2)
    Bt = sla.lu_solve(f["luA1"], Bt.reshape(n * n, n, order="F").T).T.reshape((n, n, n), order="F")
    X = np.empty_like(Bt)
    for k in range(n):
        # slice k: (T_1 (x) I + I (x) T_2) y = (Q_1^T (x) Q_2^T) b~_k
        C = f["Q2"].T @ Bt[:, :, k] @ f["Q1"]
        Y = sla.solve_sylvester(f["T2"], f["T1"].T, C)
        X[:, :, k] = f["Q2"] @ Y @ f["Q1"].T
    return X.reshape(-1, order="F")


class BlockPrecond:
    """Element-by-element P^-1 for a global vector (element-major layout)."""

    def __init__(self, nloc: int, solvers):
        self.nloc, self.solvers = nloc, solvers

    def __call__(self, v: np.ndarray) -> np.ndarray:
        out = np.empty_like(v)
        for e, solve in enumerate(self.solvers):
            s = slice(e * self.nloc, (e + 1) * self.nloc)
            out[s] = solve(v[s])
        return out


def block_jacobi(dg) -> BlockPrecond:
    """Exact block Jacobi: LU of each exact diagonal block S_e."""
    sol = []
    for e in range(dg.mesh.num_elem):
        lu = sla.lu_factor(dg.element_block(e))
        sol.append(lambda v, lu=lu: sla.lu_solve(lu, v))
    return BlockPrecond(dg.nloc, sol)


def kron_dense(dg, blocks=None, r: int = 2) -> BlockPrecond:
    """KSVD preconditioner applied by dense LU of each assembled P_e."""
    from .ksvd import ksvd_2d, ksvd_3d_nested, kron_sum
    sol = []
    for e in range(dg.mesh.num_elem):
        S = dg.element_block(e) if blocks is None else blocks[e]
        if dg.dim == 2:
            _, As, Bs = ksvd_2d(S, dg.n, r)
            P = kron_sum(As, Bs)
        else:
            P = ksvd_3d_nested(S, dg.n)["P"]
        lu = sla.lu_factor(P)
        sol.append(lambda v, lu=lu: sla.lu_solve(lu, v))
    return BlockPrecond(dg.nloc, sol)
