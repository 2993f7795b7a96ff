"""GPU parity: GMRES solves vs the oracle's GMRES and direct solves."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla
import torch

import synthetic
from oracle.gmres import gmres
from oracle.precond import block_jacobi, kron_dense
from paper_1704_04549_gb300 import (TPP_FEAT_BLOCK_JACOBI, TPP_FEAT_MIXED, TPP_FP32,
                                    TPP_PC_BLOCK_JACOBI, TPP_PC_KRON, TPP_PC_NONE)
from tests.gpu_util import make_pair, rel, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("h", [1.0, 1.0 / 8])
def test_config_8x8_constant_jacobi_vs_kron(h):
    """8x8 periodic unit-square quads (and the h = 1/8 reading), n = 8,
    a = (1, 0.5), dt = 0.1: J and K give the same iteration counts."""
    ctx, dg = make_pair(8, (8, 8), 0.1, synthetic.constant_velocity([1.0, 0.5]),
                        features=TPP_FEAT_BLOCK_JACOBI, h=h)
    ctx.tpp_build_factors()
    ctx.tpp_build_block_jacobi()
    b = synthetic.rhs(1704, dg.ndof)
    S = dg.global_matrix()
    xs = spla.spsolve(S.tocsc(), b)
    xK, rK = ctx.gmres_solve(to_dev(b), pc=TPP_PC_KRON, rtol=1e-8)
    xJ, rJ = ctx.gmres_solve(to_dev(b), pc=TPP_PC_BLOCK_JACOBI, rtol=1e-8)
    _, oK = gmres(lambda v: S @ v, b, M=kron_dense(dg), rtol=1e-8)
    _, oJ = gmres(lambda v: S @ v, b, M=block_jacobi(dg), rtol=1e-8)
    assert rK["converged"] and rJ["converged"]
    assert rK["true_rel_res"] <= 1e-8 and rJ["true_rel_res"] <= 1e-8
    assert rK["iters"] == rJ["iters"]
    assert abs(rK["iters"] - oK["iters"]) <= 1 and abs(rJ["iters"] - oJ["iters"]) <= 1
    assert rel(to_host(xK), xs) <= 1e-6 and rel(to_host(xJ), xs) <= 1e-6
    # block-Jacobi apply vs the oracle's exact block inverse
    r = synthetic.rhs(3, dg.ndof)
    assert rel(to_host(ctx.tpp_apply_block_jacobi(to_dev(r))), block_jacobi(dg)(r)) <= 1e-12


@pytest.mark.parametrize("n,nel,kmax", [(5, (3, 5), 1), (8, (4, 4), 1), (12, (4, 4), 1),
                                         (5, (6, 6), 2)])
def test_fourier_gmres_matches_oracle(n, nel, kmax):
    ctx, dg = make_pair(n, nel, 0.05, synthetic.fourier_velocity(1705, 2, kmax=kmax), h=1.0)
    ctx.tpp_build_factors()
    b = synthetic.rhs(1706, dg.ndof)
    S = dg.global_matrix()
    x_ref, o = gmres(lambda v: S @ v, b, M=kron_dense(dg), rtol=1e-8)
    assert o["converged"]
    x, r = ctx.gmres_solve(to_dev(b), pc=TPP_PC_KRON, rtol=1e-8)
    assert r["converged"] and r["true_rel_res"] <= 1e-8
    assert abs(r["iters"] - o["iters"]) <= 1
    assert rel(to_host(x), x_ref) <= 1e-6
    x12, r12 = ctx.gmres_solve(to_dev(b), pc=TPP_PC_KRON, rtol=1e-12)
    xs = spla.spsolve(S.tocsc(), b)
    assert r12["true_rel_res"] <= 1e-12 and rel(to_host(x12), xs) <= 1e-9


def test_reduced_mesh_of_the_bench_field_n16():
    """n = 16 on 16 x 16 unit-square quads with the random-Fourier field of the 64 x 64
    workload scaled by the mesh (wavenumber 1 here, 1..4 there: each element sees the
    same fraction, 1/16, of a period): iteration count equal to the oracle's +-1, both
    true residuals <= 1e-8, solution within 1e-6 of the oracle's."""
    ctx, dg = make_pair(16, (16, 16), 0.05, synthetic.fourier_velocity(1705, 2, kmax=1), h=1.0)
    ctx.tpp_build_factors()
    b = synthetic.rhs(1706, dg.ndof)
    S = dg.global_matrix()
    x_ref, o = gmres(lambda v: S @ v, b, M=kron_dense(dg), rtol=1e-8)
    x, r = ctx.gmres_solve(to_dev(b), pc=TPP_PC_KRON, rtol=1e-8)
    print(f"16x16 n=16: GPU {r['iters']} iterations, oracle {o['iters']}")
    assert o["converged"] and r["converged"] and r["true_rel_res"] <= 1e-8
    assert abs(r["iters"] - o["iters"]) <= 1
    xh = to_host(x)
    assert np.linalg.norm(b - S @ xh) <= 1.0001e-8 * np.linalg.norm(b)
    assert rel(xh, x_ref) <= 1e-6


@pytest.mark.parametrize("n,kmax,iters", [(16, 4, 90), (31, 1, 60)])
def test_stall_is_the_methods(n, kmax, iters):
    """8 x 8 unit-square quads: with wavenumbers 1..4 at n = 16, and with wavenumber 1
    at n = 31, the oracle's GMRES(30) with the exact-KSVD preconditioner stalls (no
    1e-8 within hundreds of iterations).  The GPU solver stalls alike: after the same
    number of Arnoldi steps both true residuals agree to 2%, so the stagnation is the
    preconditioner's (the method's), not the CUDA path's."""
    ctx, dg = make_pair(n, (8, 8), 0.05, synthetic.fourier_velocity(1705, 2, kmax=kmax), h=1.0)
    ctx.tpp_build_factors()
    b = synthetic.rhs(1706, dg.ndof)
    S = dg.global_matrix()
    x_ref, o = gmres(lambda v: S @ v, b, M=kron_dense(dg), rtol=1e-8, max_iters=iters)
    x, r = ctx.gmres_solve(to_dev(b), pc=TPP_PC_KRON, rtol=1e-8, max_iters=iters, check=False)
    print(f"8x8 n={n} kmax={kmax}: after {iters} steps GPU {r['true_rel_res']:.4e}, "
          f"oracle {o['true_rel_res']:.4e}")
    assert not o["converged"] and not r["converged"] and r["iters"] == o["iters"] == iters
    assert abs(r["true_rel_res"] - o["true_rel_res"]) <= 0.02 * o["true_rel_res"]
    assert o["true_rel_res"] > 1e-4
    # the GPU residual is a true residual: recomputed with the oracle's S
    assert abs(np.linalg.norm(b - S @ to_host(x)) / np.linalg.norm(b) - r["true_rel_res"]) <= \
        1e-10


def test_unpreconditioned_restarted():
    ctx, dg = make_pair(3, (3, 3), 0.05, synthetic.fourier_velocity(6, 2))
    b = synthetic.rhs(2, dg.ndof)
    S = dg.global_matrix()
    x, r = ctx.gmres_solve(to_dev(b), pc=TPP_PC_NONE, restart=5, rtol=1e-10, max_iters=5000)
    _, o = gmres(lambda v: S @ v, b, restart=5, rtol=1e-10, max_iters=5000)
    assert r["converged"] and abs(r["iters"] - o["iters"]) <= 2
    assert np.linalg.norm(S @ to_host(x) - b) <= 1e-10 * np.linalg.norm(b)


def test_zero_rhs_and_max_iters():
    ctx, dg = make_pair(4, (2, 2), 0.05, synthetic.fourier_velocity(6, 2))
    ctx.tpp_build_factors()
    import torch
    x, r = ctx.gmres_solve(torch.zeros(dg.ndof, dtype=torch.float64, device="cuda:0"))
    assert r["converged"] and r["iters"] == 0 and not to_host(x).any()
    b = synthetic.rhs(2, dg.ndof)
    x, r = ctx.gmres_solve(to_dev(b), pc=TPP_PC_NONE, max_iters=3, rtol=1e-14, check=False)
    assert r["status"] == 4 and r["iters"] == 3 and not r["converged"]


def test_full_size_fourier_n16_converges():
    """64 x 64 unit-square quads, n = 16, random-Fourier field, dt = 0.05."""
    ctx, dg = make_pair(16, (64, 64), 0.05, synthetic.fourier_velocity(1705, 2), h=1.0)
    ctx.tpp_build_factors()
    b = synthetic.rhs(1706, dg.ndof)
    x, r = ctx.gmres_solve(to_dev(b), pc=TPP_PC_KRON, rtol=1e-8)
    assert r["converged"] and r["true_rel_res"] <= 1e-8
    # residual recomputed through the operator entry point, and by the oracle's
    # sum-factorised matvec (written independently of the CUDA operator)
    Ax = to_host(ctx.dg_apply_sumfact(x))
    assert np.linalg.norm(Ax - b) <= 1.0001e-8 * np.linalg.norm(b)
    Ax_ref = dg.apply_sumfact(to_host(x))
    assert np.linalg.norm(Ax_ref - b) <= 1.0001e-8 * np.linalg.norm(b)


@pytest.mark.parametrize("n", [8, 16])
def test_mixed_precision_2d(n):
    """FP32 apply against the FP64 apply, and flexible GMRES with the FP32 inner
    preconditioner reaching the same 1e-8 true residual."""
    ctx, dg = make_pair(n, (4, 4), 0.05, synthetic.fourier_velocity(1705, 2, kmax=1),
                        features=TPP_FEAT_MIXED, h=1.0)
    ctx.tpp_build_factors()
    b = synthetic.rhs(1706, dg.ndof)
    x64 = to_host(ctx.tpp_apply_inverse(to_dev(b)))
    x32 = to_host(ctx.tpp_apply_inverse(to_dev(b), prec=TPP_FP32))
    cp = to_host(ctx.views()["cond"]).max()
    # FP32 contractions and Sylvester solve: error ~ n u32 times the factor conditioning
    assert rel(x32, x64) <= 1e-6 * n * max(1.0, np.sqrt(cp))
    _, r64 = ctx.gmres_solve(to_dev(b), pc=TPP_PC_KRON, rtol=1e-8)
    _, r32 = ctx.gmres_solve(to_dev(b), pc=TPP_PC_KRON, rtol=1e-8, inner_prec=TPP_FP32,
                             flexible=True)
    assert r32["converged"] and r32["true_rel_res"] <= 1e-8
    assert r32["iters"] <= r64["iters"] + 3


@pytest.mark.parametrize("n,nel,kin", [(8, (8, 8), 0), (8, (8, 8), 8), (5, (3, 3, 3), 0),
                                       (16, (6, 6), 12)])
def test_graph_cycles_match_plain_launches(n, nel, kin):
    """use_graph runs each group of Arnoldi steps as one captured CUDA graph: the
    same kernels in the same order, so the same iterates bit for bit; a second
    solve replays the cached graphs and a new restart length recaptures."""
    from paper_1704_04549_gb300 import TPP_FEAT_MIXED
    vel = synthetic.fourier_velocity(1705, len(nel))
    ctx, dg = make_pair(n, nel, 0.05, vel, features=TPP_FEAT_MIXED, h=1.0)
    ctx.tpp_build_factors()
    b = to_dev(synthetic.rhs(1707, dg.ndof))
    for restart in (10, 30, 10):
        kw = dict(pc=TPP_PC_KRON, rtol=1e-9, restart=restart, inner_iters=kin, max_iters=300,
                  check=False)
        x0, r0 = ctx.gmres_solve(b, **kw)
        x1, r1 = ctx.gmres_solve(b, use_graph=True, **kw)
        assert r1["converged"] == r0["converged"] and r1["status"] == r0["status"]
        assert r1["iters"] == r0["iters"] and r1["cycles"] == r0["cycles"]
        assert r1["inner_iters"] == r0["inner_iters"]
        assert torch.equal(x0, x1)
        if restart == 30 and kin == 0:
            assert r1["converged"]
