"""Pins for oracle/ksvd.py: rearrangement, Eq. NKP identity, exact recovery."""
import numpy as np
import pytest

import synthetic
from oracle.dg import AdvectionDG, PeriodicMesh
from oracle.ksvd import ksvd, ksvd_2d, ksvd_3d_nested, kron_sum, rearrange, vec


def test_rearranged_kronecker_is_outer_product_of_vecs():
    rng = np.random.default_rng(0)
    m1, n1, m2, n2 = 3, 4, 2, 5
    A, B = rng.standard_normal((m1, n1)), rng.standard_normal((m2, n2))
    At = rearrange(np.kron(A, B), m1, n1, m2, n2)
    assert np.array_equal(At, np.outer(vec(A), vec(B)))
    # brute force on the index map: entry (i*m2+a, j*n2+b) of A lands in
    # row j*m1+i, column b*m2+a of the rearranged matrix
    S = rng.standard_normal((m1 * m2, n1 * n2))
    St = rearrange(S, m1, n1, m2, n2)
    for i in range(m1):
        for j in range(n1):
            for a in range(m2):
                for b in range(n2):
                    assert St[j * m1 + i, b * m2 + a] == S[i * m2 + a, j * n2 + b]


@pytest.mark.parametrize("r", [1, 2, 3])
def test_frobenius_identity_and_optimality(r):
    rng = np.random.default_rng(r)
    n = 4
    S = rng.standard_normal((n * n, n * n))
    s, As, Bs = ksvd_2d(S, n, r)
    err = np.linalg.norm(S - kron_sum(As, Bs))
    assert abs(err - np.sqrt(np.sum(s[r:] ** 2))) < 1e-12 * np.linalg.norm(S)
    for _ in range(5):       # any perturbation of the factors is worse
        dA = [a + 1e-3 * rng.standard_normal(a.shape) for a in As]
        assert np.linalg.norm(S - kron_sum(dA, Bs)) > err


def test_exact_recovery_of_two_term_sum():
    rng = np.random.default_rng(7)
    n = 6
    A1, B1, A2, B2 = (rng.standard_normal((n, n)) for _ in range(4))
    S = np.kron(A1, B1) + np.kron(A2, B2)
    s, As, Bs = ksvd_2d(S, n)
    assert s[2] / s[0] < 1e-14
    assert np.linalg.norm(S - kron_sum(As, Bs)) < 1e-13 * np.linalg.norm(S)


def test_exact_recovery_3d_nested():
    rng = np.random.default_rng(8)
    n = 3
    A1, B1, C1, B2, C2 = (rng.standard_normal((n, n)) for _ in range(5))
    S = np.kron(A1, np.kron(B1, C1) + np.kron(B2, C2))
    out = ksvd_3d_nested(S, n)
    assert out["s1"][1] / out["s1"][0] < 1e-14
    assert out["s2"][2] / out["s2"][0] < 1e-14
    assert np.linalg.norm(S - out["P"]) < 1e-13 * np.linalg.norm(S)


@pytest.mark.parametrize("n", [2, 4, 8])
@pytest.mark.parametrize("field", ["constant", "separable"])
def test_advection_block_is_exact_two_term_sum(n, field):
    # Cartesian mesh with constant (Eq. adv-kron-const) or separable
    # (Eq. adv-kron-cart) velocity: the diagonal block is exactly
    # A_1 (x) B_1 + A_2 (x) B_2, face terms included.
    vel = (synthetic.constant_velocity([1.0, 0.5]) if field == "constant"
           else synthetic.fourier_velocity(4, 2, separable=True))
    dg = AdvectionDG(PeriodicMesh((4, 4)), n, 0.1, vel)
    for e in [0, 7]:
        S = dg.element_block(e)
        s, As, Bs = ksvd_2d(S, n)
        assert s[2] / s[0] < 1e-14 if n > 1 else True
        assert np.linalg.norm(S - kron_sum(As, Bs)) < 1e-13 * np.linalg.norm(S)


def test_nonseparable_block_is_not_exact():
    vel = synthetic.fourier_velocity(4, 2)
    dg = AdvectionDG(PeriodicMesh((4, 4)), 6, 0.5, vel)
    s, _, _ = ksvd_2d(dg.element_block(3), 6)
    assert s[2] / s[0] > 1e-6


@pytest.mark.parametrize("n", [3, 5, 8])
def test_rearranged_2d_block_has_rank_at_most_2n(n):
    # collocated quadrature: x-terms of the block carry delta_{l j}, y-terms
    # delta_{k i}, so A~ is n rows plus n columns: rank <= 2n
    dg = AdvectionDG(PeriodicMesh((3, 3)), n, 0.3, synthetic.fourier_velocity(9, 2))
    s = np.linalg.svd(rearrange(dg.element_block(4), n, n, n, n), compute_uv=False)
    assert s[2 * n] / s[0] < 1e-14
    assert s[2 * n - 1] / s[0] > 1e-14


def test_3d_constant_velocity_first_stage_not_rank_one():
    # the nested rank-1 first stage is not exact even for constant velocity
    dg = AdvectionDG(PeriodicMesh((2, 2, 2)), 3, 0.1, synthetic.constant_velocity([1.0, 0.5, 0.25]))
    s, _, _ = ksvd(dg.element_block(0), 3, 3, 9, 9, 1)
    assert s[1] / s[0] > 1e-6 and s[2] / s[0] < 1e-14


@pytest.mark.parametrize("n", [3, 4])
def test_3d_nested_stages_on_advection_blocks(n):
    """The nested construction (Sec. 4.3) on real 3D advection blocks, where neither
    stage is exact: each stage's error is the Eckart-Young tail of its rearrangement,
    a perturbed stage-1 factor is worse, and the two errors add in quadrature,
    ||S - P||^2 = ||S - A1 (x) D1||^2 + ||A1||^2 ||D1 - D1_2||^2, because the stage-1
    residual is orthogonal to every A1 (x) X (it fails when P is assembled from a
    different A1 than the one stage 2 was scaled against).  Which operator the
    stages approximate is pinned by the exact-recovery test above."""
    dg = AdvectionDG(PeriodicMesh((2, 2, 2)), n, 0.1, synthetic.fourier_velocity(11, 3))
    rng = np.random.default_rng(n)
    for e in [0, 5]:
        S = dg.element_block(e)
        out = ksvd_3d_nested(S, n)
        A1, D1, s1, s2 = out["A1"], out["D1"], out["s1"], out["s2"]
        R1 = S - np.kron(A1, D1)
        assert abs(np.linalg.norm(R1) - np.sqrt(np.sum(s1[1:] ** 2))) <= 1e-12 * np.linalg.norm(S)
        assert s1[1] / s1[0] > 1e-8                     # stage 1 is not exact
        for _ in range(3):
            dA = A1 + 1e-3 * rng.standard_normal(A1.shape)
            assert np.linalg.norm(S - np.kron(dA, D1)) > np.linalg.norm(R1)
        D12 = np.kron(out["B1"], out["C1"]) + np.kron(out["B2"], out["C2"])
        R2 = D1 - D12
        assert abs(np.linalg.norm(R2) - np.sqrt(np.sum(s2[2:] ** 2))) <= 1e-12 * np.linalg.norm(D1)
        lhs = np.linalg.norm(S - out["P"]) ** 2
        rhs = np.linalg.norm(R1) ** 2 + np.linalg.norm(A1) ** 2 * np.linalg.norm(R2) ** 2
        assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(S) ** 2
