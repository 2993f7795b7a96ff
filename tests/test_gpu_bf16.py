"""GPU: the BF16 tensor-core Kronecker apply (TPP_BF16: BF16 factors and stage inputs,
FP32 accumulation, mma.sync tensor-core tiles) against the oracle's dense solve, with
its stated error bound, and as the preconditioner of the mixed-precision solver."""
import numpy as np
import pytest

import synthetic
from oracle.dg import IsolatedElements
from oracle.ksvd import ksvd_2d, kron_sum
from oracle.precond import apply_dense
from paper_1704_04549_gb300 import (TPP_BF16, TPP_FEAT_BF16, TPP_FEAT_MIXED, TPP_FP32,
                                    TPP_PC_KRON, Context)
from tests.gpu_util import DEV, make_pair, rel, to_dev, to_host

pytestmark = pytest.mark.gpu

# Stated bound of the BF16 apply against the oracle, element by element: BF16 factors and
# stage inputs carry 2^-9 relative rounding, amplified by the conditioning of the inverted
# factor pair (the route multiplies by L_A^-1 and L_B^-1 explicitly), so
#     err <= 2^-7 sqrt(cond_1(L_A) cond_1(L_B)).
# Measured on the GB300 (40 isolated elements per n): the largest error / (2^-8 sqrt(cond))
# is 1.34 (n = 4, condition product 5.6e2, error 0.11); at n >= 8 every error is below the
# 3e-2 target (maxima 2.2e-2 at n = 8, 1.2e-2 at n = 13, 1.1e-2 at n = 16).
def bf16_bound(cond_pair):
    return 2.0 ** -7 * np.sqrt(max(cond_pair, 1.0))


BF16_TARGET = 3e-2


@pytest.mark.parametrize("n,E,R", [(4, 7, 1), (8, 5, 8), (16, 6, 19), (13, 3, 64)])
def test_bf16_apply_vs_oracle(n, E, R):
    """Isolated elements with R right-hand sides each (R = 1: one warp tile mostly padding;
    R = 19: three tiles, the last ragged; R = 64: eight tiles over four warps)."""
    rng = np.random.Generator(np.random.PCG64(40 + n))
    centres = rng.random((E, 2))
    vel = synthetic.fourier_velocity(1705, 2)
    ctx = Context(2, n, (E,), 1.0, 0.05, vel, features=TPP_FEAT_BF16, device=DEV,
                  batch_rhs=R, centres=centres, batch_span=1.0 / 64)
    iso = IsolatedElements(n, 1.0, centres, 0.05, vel, span=1.0 / 64)
    ctx.tpp_build_factors()
    nl = n * n
    b = synthetic.rhs(5 + n, E * R * nl)
    x16 = to_host(ctx.tpp_apply_inverse(to_dev(b), prec=TPP_BF16)).reshape(E, R, nl)
    x64 = to_host(ctx.tpp_apply_inverse(to_dev(b))).reshape(E, R, nl)
    B = b.reshape(E, R, nl)
    cp = to_host(ctx.views()["cond"])
    worst = 0.0
    for e in range(E):
        _, As, Bs = ksvd_2d(iso.block(e), n)
        P = kron_sum(As, Bs)
        for r in range(R):
            ref = apply_dense(P, B[e, r])
            err = rel(x16[e, r], ref)
            worst = max(worst, err)
            assert err <= bf16_bound(cp[e]), (e, r, err, cp[e])
            if n >= 8:
                assert err <= BF16_TARGET, (e, r, err)
            assert rel(x64[e, r], ref) <= 1e-10
    print(f"BF16 apply vs oracle, n={n} R={R}: max element relative error {worst:.2e}")


def test_bf16_apply_on_a_mesh():
    """Coupled 4 x 4 mesh at n = 16 (one right-hand side per element, the warp tile
    mostly padding): the BF16 apply stays within its bounds of the FP64 apply."""
    ctx, dg = make_pair(16, (4, 4), 0.05, synthetic.fourier_velocity(1705, 2),
                        features=TPP_FEAT_BF16, h=1.0)
    ctx.tpp_build_factors()
    b = to_dev(synthetic.rhs(11, dg.ndof))
    x16 = to_host(ctx.tpp_apply_inverse(b, prec=TPP_BF16)).reshape(16, 256)
    x64 = to_host(ctx.tpp_apply_inverse(b)).reshape(16, 256)
    cp = to_host(ctx.views()["cond"])
    for e in range(16):
        assert rel(x16[e], x64[e]) <= min(BF16_TARGET, bf16_bound(cp[e]))


@pytest.mark.parametrize("kin", [0, 12])
def test_bf16_preconditioned_solver_reaches_fp64_residual(kin):
    """Flexible FP64 GMRES with the BF16 apply (kin = 0), and FP64 FGMRES around inner
    FP32 GMRES(12) preconditioned by the BF16 apply: the 1e-8 true FP64 residual."""
    ctx, dg = make_pair(16, (8, 8), 0.05, synthetic.fourier_velocity(1705, 2, kmax=1),
                        features=TPP_FEAT_BF16 | TPP_FEAT_MIXED, h=1.0)
    ctx.tpp_build_factors()
    b = synthetic.rhs(1706, dg.ndof)
    _, r64 = ctx.gmres_solve(to_dev(b), pc=TPP_PC_KRON, rtol=1e-8)
    x, r = ctx.gmres_solve(to_dev(b), pc=TPP_PC_KRON, rtol=1e-8, inner_prec=TPP_BF16,
                           flexible=True, inner_iters=kin)
    print(f"BF16 preconditioner, inner {kin}: {r['iters']} outer iterations "
          f"(FP64: {r64['iters']}), {r['inner_iters']} inner")
    assert r["converged"] and r["true_rel_res"] <= 1e-8
    if kin == 0:
        assert r["iters"] <= r64["iters"] + 6
    S = dg.global_matrix()
    assert np.linalg.norm(b - S @ to_host(x)) <= 1.0001e-8 * np.linalg.norm(b)
