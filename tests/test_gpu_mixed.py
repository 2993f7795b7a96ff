"""GPU: the FP32 forms of the operator and the Kronecker apply (stated error
bounds against the FP64 oracle / FP64 path), and the mixed-precision solver
(FP64 flexible GMRES around inner FP32 GMRES solves)."""
import numpy as np
import pytest
import torch

import synthetic
from paper_1704_04549_gb300 import TPP_FEAT_MIXED, TPP_FP32, TPP_PC_KRON
from tests.gpu_util import make_pair, rel, to_dev, to_host

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24


def _vel(dim, kmax=4):
    return synthetic.fourier_velocity(1705, dim, kmax=kmax)


@pytest.mark.parametrize("n,nel", [(3, (3, 4)), (8, (4, 4)), (16, (3, 3)), (31, (2, 2)),
                                   (4, (2, 3, 2)), (11, (2, 2, 2))])
def test_operator_f32_within_rounding_bound(n, nel):
    """|y32 - S x| <= (3n + 10) u32 (|S| |x|) entrywise: each output is a sum of at
    most 3n + 10 rounded products of rounded inputs (first-order bound)."""
    ctx, dg = make_pair(n, nel, 0.05, _vel(len(nel)), features=TPP_FEAT_MIXED)
    S = dg.global_matrix()
    x = synthetic.rhs(7, dg.ndof).astype(np.float32)
    y32 = to_host(ctx.dg_apply_sumfact_f32(torch.as_tensor(x, device="cuda:0")))
    xd = x.astype(np.float64)
    y = S @ xd
    bound = (3 * n + 10) * U32 * (abs(S) @ np.abs(xd))
    assert np.all(np.abs(y32 - y) <= bound + 1e-300)


@pytest.mark.parametrize("n,nel", [(8, (4, 4)), (16, (4, 4)), (6, (2, 2, 2))])
def test_apply_f32_vs_fp64(n, nel):
    ctx, dg = make_pair(n, nel, 0.05, _vel(len(nel)), features=TPP_FEAT_MIXED)
    ctx.tpp_build_factors()
    b = synthetic.rhs(99, dg.ndof)
    x64 = to_host(ctx.tpp_apply_inverse(to_dev(b)))
    x32 = to_host(ctx.tpp_apply_inverse_f32(torch.as_tensor(b.astype(np.float32), device="cuda:0")))
    xd = to_host(ctx.tpp_apply_inverse(to_dev(b), prec=TPP_FP32))
    cp = to_host(ctx.views()["cond"]).max()
    # FP32 contractions and sweep: error ~ n u32 times the factor conditioning
    assert rel(x32, x64) <= 1e-6 * n * max(1.0, np.sqrt(cp))
    # float or double vectors around the same FP32 factors agree to input rounding
    assert rel(x32, xd) <= 1e-6 * n * max(1.0, np.sqrt(cp))


@pytest.mark.parametrize("n,nel,kmax,kin", [(8, (4, 4), 1, 8), (16, (4, 4), 1, 12),
                                            (16, (64, 64), 4, 16), (5, (3, 3, 3), 4, 10),
                                            (11, (16, 16, 16), 1, 16)])
def test_nested_mixed_gmres_reaches_fp64_residual(n, nel, kmax, kin):
    """Outer FP64 flexible GMRES with inner FP32 GMRES(kin) solves reaches the
    same 1e-8 true residual (FP64 operator) as the FP64 solver."""
    ctx, dg = make_pair(n, nel, 0.05, _vel(len(nel), kmax), features=TPP_FEAT_MIXED, h=1.0)
    ctx.tpp_build_factors()
    b = synthetic.rhs(1706, dg.ndof)
    _, r64 = ctx.gmres_solve(to_dev(b), pc=TPP_PC_KRON, rtol=1e-8)
    x, r = ctx.gmres_solve(to_dev(b), pc=TPP_PC_KRON, rtol=1e-8, inner_iters=kin)
    assert r["converged"] and r["true_rel_res"] <= 1e-8
    assert r["inner_iters"] <= r["iters"] * kin and r["iters"] <= max(4, r64["iters"] // 4)
    Ax = to_host(ctx.dg_apply_sumfact(x))
    assert np.linalg.norm(Ax - b) <= 1.0001e-8 * np.linalg.norm(b)
