"""Kronecker-product SVD of element blocks (oracle; test infrastructure).

Sec. 4.1: the nearest Kronecker product problem (Eq. NKP) is solved by the
Van Loan-Pitsianis rearrangement A -> A~ and a truncated SVD of A~:
vec(A_k) = sqrt(sigma_k) U_k, vec(B_k) = sqrt(sigma_k) V_k, vec stacking
columns.  This module forms A~ explicitly and calls LAPACK's dense SVD
(numpy.linalg.svd); the paper's Lanczos route (Alg. lanczos) reaches the same
triplets and is what the CUDA path follows.

Rearrangement: A (m1 m2 x n1 n2) is viewed as an m1 x n1 grid of m2 x n2 blocks
A_ij; row j*m1 + i of A~ is vec(A_ij)^T (0-based), so that
||A - sum A_k (x) B_k||_F = ||A~ - sum vec(A_k) vec(B_k)^T||_F.

3D (Sec. 4.3, Alg. 3d-form): stage 1 takes the best rank-1 A ~ A_1 (x) D_1
with A_1 (n x n, slowest direction z) and D_1 (n^2 x n^2); stage 2 takes the
best rank-2 D_1 ~ B_1 (x) C_1 + B_2 (x) C_2 (B: y, C: x).

Pinned in tests/test_oracle_ksvd.py: rearrangement of a Kronecker product is
the outer product of the vecs, the Frobenius identity and optimality of the
truncation, exact recovery of synthetic two-term sums, and exact recovery of
advection blocks with constant or separable velocity on Cartesian meshes
(Eqs. adv-kron-cart, adv-kron-const).
"""
from __future__ import annotations

import numpy as np


def vec(M: np.ndarray) -> np.ndarray:
    """Stack the columns of M."""
    return M.reshape(-1, order="F")


def unvec(v: np.ndarray, m: int, n: int) -> np.ndarray:
    return v.reshape((m, n), order="F")


def rearrange(A: np.ndarray, m1: int, n1: int, m2: int, n2: int) -> np.ndarray:
    """A~ (m1 n1 x m2 n2) with row j*m1 + i equal to vec(A_ij)^T."""
    assert A.shape == (m1 * m2, n1 * n2)
    At = np.empty((m1 * n1, m2 * n2))
    for j in range(n1):
        for i in range(m1):
            blk = A[i * m2:(i + 1) * m2, j * n2:(j + 1) * n2]
            At[j * m1 + i, :] = vec(blk)
    return At


def ksvd(A: np.ndarray, m1: int, n1: int, m2: int, n2: int, r: int):
    """Best rank-r Kronecker sum sum_k A_k (x) B_k in the Frobenius norm.

    Returns (sigma_all, [A_k], [B_k]) with sigma_all all singular values of A~."""
    At = rearrange(A, m1, n1, m2, n2)
    U, s, Vt = np.linalg.svd(At)
    As, Bs = [], []
    for k in range(r):
        sk = np.sqrt(s[k]) if k < s.shape[0] else 0.0
        uk = U[:, k] if k < U.shape[1] else np.zeros(m1 * n1)
        vk = Vt[k, :] if k < Vt.shape[0] else np.zeros(m2 * n2)
        As.append(sk * unvec(uk, m1, n1))
        Bs.append(sk * unvec(vk, m2, n2))
    return s, As, Bs


def kron_sum(As, Bs) -> np.ndarray:
    return sum(np.kron(a, b) for a, b in zip(As, Bs))


def ksvd_2d(S: np.ndarray, n: int, r: int = 2):
    """Rank-r KSVD of a 2D element block (n^2 x n^2): A_k act on y, B_k on x."""
    return ksvd(S, n, n, n, n, r)


def ksvd_3d_nested(S: np.ndarray, n: int):
    """Two-stage nested KSVD of a 3D element block (n^3 x n^3), Alg. 3d-form.

    Returns dict with A1, B1, C1, B2, C2, the stage singular values s1, s2 and
    P = A1 (x) (B1 (x) C1 + B2 (x) C2)."""
    s1, (A1,), (D1,) = ksvd(S, n, n, n * n, n * n, 1)
    s2, (B1, B2), (C1, C2) = ksvd(D1, n, n, n, n, 2)
    P = np.kron(A1, np.kron(B1, C1) + np.kron(B2, C2))
    return dict(A1=A1, D1=D1, B1=B1, C1=C1, B2=B2, C2=C2, s1=s1, s2=s2, P=P)
