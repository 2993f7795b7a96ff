"""GPU parity: the coupled 2D Euler system linearised around the vortex of Sec. 5.3
(tpp_create_system) against the oracle's assembled system (oracle/systems.py): the
coupled operator, the small-block Kronecker factors and their apply, exact small-block
Jacobi, and GMRES with both small-block preconditioners."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import synthetic
from oracle.gmres import gmres
from oracle.ksvd import kron_sum, ksvd_2d
from oracle.precond import apply_dense
from oracle.systems import vortex_system
from paper_1704_04549_gb300 import (TPP_FEAT_BLOCK_JACOBI, TPP_FEAT_TWO_SIDED,
                                    TPP_PC_BLOCK_JACOBI, TPP_PC_KRON)
from tests.gpu_util import DEV, FP64_TOL, rel, solve_tol, to_dev, to_host

pytestmark = pytest.mark.gpu


def _state(n, nel, h):
    """Vortex state at the Gauss-Legendre nodes, [E][4][n^2] (x fastest, element index
    x fastest), from the input generator."""
    xg = 0.5 * (np.polynomial.legendre.leggauss(n)[0] + 1.0)
    E = nel[0] * nel[1]
    out = np.empty((E, 4, n * n))
    for e in range(E):
        cx, cy = e % nel[0], e // nel[0]
        X = np.stack(np.meshgrid((cx + xg) * h, (cy + xg) * h, indexing="xy"), -1).reshape(-1, 2)
        out[e] = synthetic.euler_vortex_state(X).T
    return out


def _pair(n, nel, h, dt, features=0):
    from paper_1704_04549_gb300 import Context
    U0 = _state(n, nel, h)
    ora = vortex_system(nel, h, n, dt, synthetic.euler_vortex_state)
    ora.U0 = U0
    ctx = Context.euler_system(n, nel, h, dt, U0, features=features, device=DEV)
    return ctx, ora


CASES = [(2, (3, 2), 5.0), (4, (4, 3), 2.5), (8, (4, 4), 2.5), (16, (2, 2), 5.0),
         (31, (2, 1), 5.0)]


@pytest.mark.parametrize("n,nel,h", CASES)
def test_coupled_operator_matches_oracle(n, nel, h):
    ctx, ora = _pair(n, nel, h, 0.1)
    S = ora.global_matrix()
    x = synthetic.rhs(7, ora.ndof)
    y = to_host(ctx.dg_apply_sumfact(to_dev(x)))
    assert rel(y, S @ x) <= FP64_TOL, rel(y, S @ x)
    if n <= 16:
        ys = to_host(ctx.dg_apply_sumfact_static(to_dev(x)))
        assert rel(ys, S @ x) <= FP64_TOL


@pytest.mark.parametrize("n,nel,h", CASES[:4])
@pytest.mark.parametrize("form", ["one-sided", "two-sided"])
def test_small_block_factors_apply_and_jacobi(n, nel, h, form):
    feats = TPP_FEAT_BLOCK_JACOBI | (TPP_FEAT_TWO_SIDED if form == "two-sided" else 0)
    ctx, ora = _pair(n, nel, h, 0.1, features=feats)
    rep = ctx.tpp_build_factors()
    assert rep["num_schur_fail"] == 0
    ctx.tpp_build_block_jacobi()
    v = ctx.views()
    sig = to_host(v["sigma"])
    A1, B1, A2, B2 = (to_host(v[k]) for k in ("A1", "B1", "A2", "B2"))
    cpair = to_host(v["cond"])
    b = synthetic.rhs(9, ora.ndof)
    xk = to_host(ctx.tpp_apply_inverse(to_dev(b)))
    xj = to_host(ctx.tpp_apply_block_jacobi(to_dev(b)))
    nl = ora.nloc
    for e in range(ora.mesh.num_elem):
        for c in range(4):
            k = e * 4 + c
            Ssm = ora.small_block(e, c)
            s_ref, As, Bs = ksvd_2d(Ssm, n)
            P_ref = kron_sum(As, Bs)
            assert abs(sig[k, 0] - s_ref[0]) <= FP64_TOL * s_ref[0]
            P = np.kron(A1[k], B1[k]) + np.kron(A2[k], B2[k])
            assert rel(P, P_ref) <= FP64_TOL, (e, c, rel(P, P_ref))
            blk = slice(k * nl, (k + 1) * nl)
            err = rel(xk[blk], apply_dense(P_ref, b[blk]))
            assert err <= solve_tol(np.linalg.cond(P_ref), cpair[k]), (e, c, err)
            assert rel(xj[blk], np.linalg.solve(Ssm, b[blk])) <= FP64_TOL * np.linalg.cond(Ssm)


def _oracle_precond(ora, kind):
    nl, inv = ora.nloc, []
    for e in range(ora.mesh.num_elem):
        for c in range(4):
            Ssm = ora.small_block(e, c)
            if kind == "K":
                _, As, Bs = ksvd_2d(Ssm, ora.n)
                inv.append(np.linalg.inv(kron_sum(As, Bs)))
            else:
                inv.append(np.linalg.inv(Ssm))

    def apply(v):
        out = np.empty_like(v)
        for k, Pi in enumerate(inv):
            out[k * nl:(k + 1) * nl] = Pi @ v[k * nl:(k + 1) * nl]
        return out
    return apply


@pytest.mark.parametrize("n,nel,h,dt", [(4, (4, 3), 2.5, 0.1), (8, (4, 4), 2.5, 0.1),
                                         (8, (4, 4), 2.5, 0.01), (12, (3, 3), 2.5, 0.1)])
def test_gmres_with_small_block_preconditioners(n, nel, h, dt):
    ctx, ora = _pair(n, nel, h, dt, features=TPP_FEAT_BLOCK_JACOBI)
    ctx.tpp_build_factors()
    ctx.tpp_build_block_jacobi()
    S = ora.global_matrix()
    b = synthetic.rhs(11, ora.ndof)
    xs = spla.spsolve(S.tocsc(), b)
    its = {}
    for kind, pc in (("K", TPP_PC_KRON), ("J", TPP_PC_BLOCK_JACOBI)):
        x_ref, o = gmres(lambda v: S @ v, b, M=_oracle_precond(ora, kind), rtol=1e-8)
        assert o["converged"]
        x, r = ctx.gmres_solve(to_dev(b), pc=pc, rtol=1e-8)
        assert r["converged"] and r["true_rel_res"] <= 1e-8
        xh = to_host(x)
        assert np.linalg.norm(b - S @ xh) <= 1.0001e-8 * np.linalg.norm(b)
        assert abs(r["iters"] - o["iters"]) <= 1, (kind, r["iters"], o["iters"])
        assert rel(xh, xs) <= 1e-6
        its[kind] = (r["iters"], o["iters"])
    print(f"Euler vortex n={n} dt={dt}: GMRES(30) iterations (GPU, oracle) K_small {its['K']}, "
          f"J_small {its['J']}")


def test_nearly_defective_density_blocks():
    """Away from the vortex the density component's small block is the mass plus face
    terms only, and its factor pencil has an eigenvalue of multiplicity n - 2 that the
    Francis iteration cannot resolve to eps: those elements are deflated at sqrt(eps)
    (flags bit 4).  The apply then matches the oracle's P^-1 b to sqrt(eps)-level
    accuracy, and GMRES still converges with the oracle's iteration count."""
    n, nel, h, dt = 8, (16, 12), 1.25, 0.1
    ctx, ora = _pair(n, nel, h, dt)
    rep = ctx.tpp_build_factors()
    assert rep["num_schur_fail"] == 0 and rep["num_schur_relaxed"] > 0
    flags = to_host(ctx.views()["flags"])
    relaxed = np.nonzero(flags & 16)[0]
    assert len(relaxed) == rep["num_schur_relaxed"] and np.all(relaxed % 4 == 0)
    b = synthetic.rhs(13, ora.ndof)
    x = to_host(ctx.tpp_apply_inverse(to_dev(b)))
    nl = ora.nloc
    worst = 0.0
    for k in relaxed[:12]:
        e, c = divmod(int(k), 4)
        _, As, Bs = ksvd_2d(ora.small_block(e, c), n)
        P = kron_sum(As, Bs)
        err = rel(x[k * nl:(k + 1) * nl], apply_dense(P, b[k * nl:(k + 1) * nl]))
        worst = max(worst, err)
        assert err <= 1.5e-8 * np.linalg.cond(P) * 10, (k, err)
    S = ora.global_matrix()
    _, o = gmres(lambda v: S @ v, b, M=_oracle_precond(ora, "K"), rtol=1e-8)
    xg, r = ctx.gmres_solve(to_dev(b), pc=TPP_PC_KRON, rtol=1e-8)
    assert r["converged"] and abs(r["iters"] - o["iters"]) <= 1
    assert np.linalg.norm(b - S @ to_host(xg)) <= 1.0001e-8 * np.linalg.norm(b)
    print(f"relaxed Schur deflation on {len(relaxed)} density blocks; worst apply error "
          f"{worst:.1e}; GMRES {r['iters']} (oracle {o['iters']})")


# ---- full blocks (Sec. 5.3: A_k of size n_c (p+1), B_k of size p+1) ------------------
FULL_CASES = [(2, (3, 2), 5.0), (3, (3, 3), 2.5), (4, (4, 3), 2.5), (8, (4, 4), 2.5),
              (16, (2, 2), 5.0)]


@pytest.mark.parametrize("n,nel,h", FULL_CASES)
def test_full_block_factors_apply_and_jacobi(n, nel, h):
    """K_full and J_full: the factors of every element's whole n_c n^2 block against the
    oracle's rank-2 KSVD with the (component, y) x (x) split, their inverse, and the exact
    full-block LU."""
    from paper_1704_04549_gb300 import TPP_FEAT_FULL_BLOCKS
    ctx, ora = _pair(n, nel, h, 0.1, features=TPP_FEAT_FULL_BLOCKS | TPP_FEAT_BLOCK_JACOBI)
    rep = ctx.tpp_build_factors()
    assert rep["num_schur_fail"] == 0
    ctx.tpp_build_block_jacobi()
    v = ctx.views()
    fA, fB, fsig = to_host(v["fA"]), to_host(v["fB"]), to_host(v["fsig"])
    fflags = to_host(v["fflags"])
    b = synthetic.rhs(19, ora.ndof)
    xk = to_host(ctx.tpp_apply_inverse(to_dev(b)))
    xj = to_host(ctx.tpp_apply_block_jacobi(to_dev(b)))
    bs = ora.bs
    worst_P, worst_x = 0.0, 0.0
    for e in range(ora.mesh.num_elem):
        s_ref, As, Bs = ora.full_block_ksvd(e)
        assert abs(fsig[e, 0] - s_ref[0]) <= 1e-12 * s_ref[0], (e, fsig[e], s_ref[:2])
        assert abs(fsig[e, 1] - s_ref[1]) <= 1e-12 * s_ref[0], (e, fsig[e], s_ref[:2])
        P_ref = kron_sum(As, Bs)
        P = np.kron(fA[e, 0], fB[e, 0]) + np.kron(fA[e, 1], fB[e, 1])
        worst_P = max(worst_P, rel(P, P_ref))
        assert rel(P, P_ref) <= 1e-13, (e, rel(P, P_ref))     # measured <= 1.1e-14
        blk = slice(e * bs, (e + 1) * bs)
        err = rel(xk[blk], np.linalg.solve(P_ref, b[blk]))
        worst_x = max(worst_x, err)
        assert err <= solve_tol(np.linalg.cond(P_ref)), (e, err)
        Se = ora.element_block(e)
        assert rel(xj[blk], np.linalg.solve(Se, b[blk])) <= FP64_TOL * np.linalg.cond(Se)
        assert fflags[e] & 12 == 0
    print(f"full blocks n={n}: max relative error of P {worst_P:.1e}, of P^-1 b {worst_x:.1e}")


@pytest.mark.parametrize("n,nel,h,dt", [(4, (4, 3), 2.5, 0.1), (8, (4, 4), 2.5, 0.1),
                                         (8, (4, 4), 2.5, 0.01), (12, (3, 3), 2.5, 0.1)])
def test_gmres_with_full_block_preconditioners(n, nel, h, dt):
    """GMRES iteration counts with K_full and J_full equal to the oracle's (+-1)."""
    from paper_1704_04549_gb300 import TPP_FEAT_FULL_BLOCKS
    ctx, ora = _pair(n, nel, h, dt, features=TPP_FEAT_FULL_BLOCKS | TPP_FEAT_BLOCK_JACOBI)
    ctx.tpp_build_factors()
    ctx.tpp_build_block_jacobi()
    S = ora.global_matrix()
    b = synthetic.rhs(11, ora.ndof)
    bs = ora.bs
    its = {}
    for kind, pc in (("K", TPP_PC_KRON), ("J", TPP_PC_BLOCK_JACOBI)):
        inv = []
        for e in range(ora.mesh.num_elem):
            if kind == "K":
                _, As, Bs = ora.full_block_ksvd(e)
                inv.append(np.linalg.inv(kron_sum(As, Bs)))
            else:
                inv.append(np.linalg.inv(ora.element_block(e)))

        def M(vec, inv=inv):
            out = np.empty_like(vec)
            for k, Pi in enumerate(inv):
                out[k * bs:(k + 1) * bs] = Pi @ vec[k * bs:(k + 1) * bs]
            return out
        _, o = gmres(lambda vec: S @ vec, b, M=M, rtol=1e-8)
        x, r = ctx.gmres_solve(to_dev(b), pc=pc, rtol=1e-8)
        assert o["converged"] and r["converged"]
        assert np.linalg.norm(b - S @ to_host(x)) <= 1.0001e-8 * np.linalg.norm(b)
        assert abs(r["iters"] - o["iters"]) <= 1, (kind, r["iters"], o["iters"])
        its[kind] = (r["iters"], o["iters"])
    print(f"Euler vortex n={n} dt={dt}: GMRES(30) iterations (GPU, oracle) K_full {its['K']}, "
          f"J_full {its['J']}")


# ---- 3D: five components (Sec. 5.6's periodic Euler case) -----------------------------
def _state3d(n, nel, h, L):
    xg = 0.5 * (np.polynomial.legendre.leggauss(n)[0] + 1.0)
    E = nel[0] * nel[1] * nel[2]
    out = np.empty((E, 5, n ** 3))
    gz, gy, gx = np.meshgrid(xg, xg, xg, indexing="ij")          # x fastest when flattened
    for e in range(E):
        cx, cy, cz = e % nel[0], (e // nel[0]) % nel[1], e // (nel[0] * nel[1])
        X = np.stack([(cx + gx) * h, (cy + gy) * h, (cz + gz) * h], -1).reshape(-1, 3)
        out[e] = synthetic.euler3d_wave_state(X, L).T
    return out


def _pair3d(n, nel, dt, features=0):
    from paper_1704_04549_gb300 import Context
    L = 2.0
    h = L / nel[0]
    U0 = _state3d(n, nel, h, L)
    ora = vortex_system(nel, h, n, dt, lambda X: synthetic.euler3d_wave_state(X, L))
    ora.U0 = U0
    ctx = Context.euler_system(n, nel, h, dt, U0, features=features, device=DEV)
    return ctx, ora


@pytest.mark.parametrize("n,nel", [(2, (2, 2, 2)), (3, (2, 2, 2)), (5, (2, 2, 2)), (8, (2, 2, 1)),
                                   (12, (2, 1, 1))])
def test_coupled_3d_operator_matches_oracle(n, nel):
    ctx, ora = _pair3d(n, nel, 0.05)
    S = ora.global_matrix()
    x = synthetic.rhs(7, ora.ndof)
    y = to_host(ctx.dg_apply_sumfact(to_dev(x)))
    assert rel(y, S @ x) <= FP64_TOL, rel(y, S @ x)


@pytest.mark.parametrize("n,nel", [(3, (2, 2, 2)), (5, (2, 2, 2))])
def test_3d_small_block_factors_and_gmres(n, nel):
    """The nested 3D KSVD (Sec. 4.3) of every small block against the oracle's, and GMRES
    on the coupled system with the small-block preconditioner (iteration parity)."""
    from oracle.ksvd import ksvd_3d_nested
    ctx, ora = _pair3d(n, nel, 0.05, features=TPP_FEAT_BLOCK_JACOBI)
    rep = ctx.tpp_build_factors()
    assert rep["num_schur_fail"] == 0
    ctx.tpp_build_block_jacobi()
    xj = to_host(ctx.tpp_apply_block_jacobi(to_dev(synthetic.rhs(9, ora.ndof))))
    v = ctx.views()
    Az = to_host(v["Az"])
    A1, B1, A2, B2 = (to_host(v[k]) for k in ("A1", "B1", "A2", "B2"))
    sigz, cpair = to_host(v["sigz"]), to_host(v["cond"])
    b = synthetic.rhs(9, ora.ndof)
    x = to_host(ctx.tpp_apply_inverse(to_dev(b)))
    nl = ora.nloc
    Ps = []
    for e in range(ora.mesh.num_elem):
        for c in range(5):
            k = e * 5 + c
            ref = ksvd_3d_nested(ora.small_block(e, c), n)
            s1 = np.atleast_1d(ref["s1"])[0]
            assert abs(sigz[k] - s1) <= 1e-12 * s1, (e, c, sigz[k], s1)
            P = np.kron(Az[k], np.kron(A1[k], B1[k]) + np.kron(A2[k], B2[k]))
            assert rel(P, ref["P"]) <= 1e-12, (e, c, rel(P, ref["P"]))
            Ps.append(ref["P"])
            xr = np.linalg.solve(ref["P"], b[k * nl:(k + 1) * nl])
            err = rel(x[k * nl:(k + 1) * nl], xr)
            assert err <= solve_tol(np.linalg.cond(ref["P"]), cpair[k] * np.linalg.cond(Az[k], 1)), (e, c, err)
            Ssm = ora.small_block(e, c)                       # J_small in 3D
            assert rel(xj[k * nl:(k + 1) * nl], np.linalg.solve(Ssm, b[k * nl:(k + 1) * nl])) <= \
                FP64_TOL * np.linalg.cond(Ssm)

    def M(vec):
        out = np.empty_like(vec)
        for k, P in enumerate(Ps):
            out[k * nl:(k + 1) * nl] = np.linalg.solve(P, vec[k * nl:(k + 1) * nl])
        return out
    S = ora.global_matrix()
    _, o = gmres(lambda vec: S @ vec, b, M=M, rtol=1e-8)
    xg, r = ctx.gmres_solve(to_dev(b), pc=TPP_PC_KRON, rtol=1e-8)
    assert o["converged"] and r["converged"] and abs(r["iters"] - o["iters"]) <= 1
    assert np.linalg.norm(b - S @ to_host(xg)) <= 1.0001e-8 * np.linalg.norm(b)
    print(f"3D Euler n={n}: GMRES K_small {r['iters']} (oracle {o['iters']})")


@pytest.mark.parametrize("n,nel", [(2, (2, 2, 2)), (3, (2, 2, 2)), (5, (2, 2, 1))])
def test_3d_full_block_jacobi(n, nel):
    """J_full in 3D (Sec. 5.6, the 5 (p+1)^3 blocks): exact LU of every element's whole
    block against a dense solve with the oracle's, and GMRES iteration parity."""
    from paper_1704_04549_gb300 import TPP_FEAT_FULL_BLOCKS
    ctx, ora = _pair3d(n, nel, 0.05, features=TPP_FEAT_FULL_BLOCKS | TPP_FEAT_BLOCK_JACOBI)
    ctx.tpp_build_block_jacobi()
    b = synthetic.rhs(23, ora.ndof)
    x = to_host(ctx.tpp_apply_block_jacobi(to_dev(b)))
    bs = ora.bs
    inv = []
    for e in range(ora.mesh.num_elem):
        Se = ora.element_block(e)
        blk = slice(e * bs, (e + 1) * bs)
        assert rel(x[blk], np.linalg.solve(Se, b[blk])) <= FP64_TOL * np.linalg.cond(Se), e
        inv.append(np.linalg.inv(Se))

    def M(vec):
        out = np.empty_like(vec)
        for k, Pi in enumerate(inv):
            out[k * bs:(k + 1) * bs] = Pi @ vec[k * bs:(k + 1) * bs]
        return out
    S = ora.global_matrix()
    _, o = gmres(lambda vec: S @ vec, b, M=M, rtol=1e-8)
    xg, r = ctx.gmres_solve(to_dev(b), pc=TPP_PC_BLOCK_JACOBI, rtol=1e-8)
    assert o["converged"] and r["converged"] and abs(r["iters"] - o["iters"]) <= 1
    assert np.linalg.norm(b - S @ to_host(xg)) <= 1.0001e-8 * np.linalg.norm(b)
    print(f"3D Euler n={n}: GMRES J_full {r['iters']} (oracle {o['iters']})")


@pytest.mark.parametrize("n,nel", [(2, (2, 2, 2)), (3, (2, 2, 2)), (5, (2, 2, 1)), (8, (2, 1, 1))])
def test_3d_full_block_factors_and_gmres(n, nel):
    """K_full in 3D: the first-stage factor A_1 (size 5n, power iteration), the y-x factors
    of D_1 and the nested P of every element against the oracle's nested KSVD of the
    whole block, P^-1 b, and GMRES iteration parity."""
    from paper_1704_04549_gb300 import TPP_FEAT_FULL_BLOCKS
    ctx, ora = _pair3d(n, nel, 0.05, features=TPP_FEAT_FULL_BLOCKS)
    rep = ctx.tpp_build_factors()
    assert rep["num_schur_fail"] == 0 and rep["num_z_unconverged"] == 0
    v = ctx.views()
    Ep = ora.mesh.num_elem
    fA, fsig, fflags = to_host(v["fA"]), to_host(v["fsig"]), to_host(v["fflags"])
    A1, B1, A2, B2 = (to_host(v[k])[:Ep] for k in ("A1", "B1", "A2", "B2"))
    b = synthetic.rhs(29, ora.ndof)
    x = to_host(ctx.tpp_apply_inverse(to_dev(b)))
    bs = ora.bs
    Ps, worst = [], 0.0
    for e in range(Ep):
        ref = ora.full_block_ksvd_3d(e)
        s1 = np.atleast_1d(ref["s1"])[0]
        assert abs(fsig[e, 0] - s1) <= 1e-12 * s1, (e, fsig[e], s1)
        P = np.kron(fA[e], np.kron(A1[e], B1[e]) + np.kron(A2[e], B2[e]))
        worst = max(worst, rel(P, ref["P"]))
        assert rel(P, ref["P"]) <= 2e-13, (e, rel(P, ref["P"]))        # measured <= 1.8e-14
        blk = slice(e * bs, (e + 1) * bs)
        err = rel(x[blk], np.linalg.solve(ref["P"], b[blk]))
        assert err <= solve_tol(np.linalg.cond(ref["P"])), (e, err)
        assert fflags[e] & 9 == 0
        Ps.append(np.linalg.inv(ref["P"]))

    def M(vec):
        out = np.empty_like(vec)
        for k, Pi in enumerate(Ps):
            out[k * bs:(k + 1) * bs] = Pi @ vec[k * bs:(k + 1) * bs]
        return out
    S = ora.global_matrix()
    _, o = gmres(lambda vec: S @ vec, b, M=M, rtol=1e-8)
    xg, r = ctx.gmres_solve(to_dev(b), pc=TPP_PC_KRON, rtol=1e-8)
    assert o["converged"] and r["converged"] and abs(r["iters"] - o["iters"]) <= 1
    assert np.linalg.norm(b - S @ to_host(xg)) <= 1.0001e-8 * np.linalg.norm(b)
    print(f"3D Euler n={n}: K_full P error {worst:.1e}, power iterations {int(fsig[:, 1].max())}, "
          f"GMRES {r['iters']} (oracle {o['iters']})")


@pytest.mark.parametrize("dim,n", [(2, 1), (2, 5), (3, 1), (3, 4)])
def test_full_blocks_degenerate_cases(dim, n):
    """dt = 0: every full block is the mass alone, an exact single Kronecker product, so the
    full-block preconditioner is exact (P^-1 b = S^-1 b); n = 1: one node per element
    (D = 0, the face terms only)."""
    from paper_1704_04549_gb300 import TPP_FEAT_FULL_BLOCKS
    for dt in (0.0, 0.05):
        if dim == 2:
            ctx, ora = _pair(n, (3, 2), 5.0, dt, features=TPP_FEAT_FULL_BLOCKS)
        else:
            ctx, ora = _pair3d(n, (2, 2, 2), dt, features=TPP_FEAT_FULL_BLOCKS)
        rep = ctx.tpp_build_factors()
        assert rep["num_schur_fail"] == 0
        b = synthetic.rhs(41, ora.ndof)
        x = to_host(ctx.tpp_apply_inverse(to_dev(b)))
        bs = ora.bs
        for e in range(ora.mesh.num_elem):
            blk = slice(e * bs, (e + 1) * bs)
            if dt == 0.0:
                Se = ora.element_block(e)
                assert rel(x[blk], np.linalg.solve(Se, b[blk])) <= 1e-13, (dt, e)
            else:
                P = (kron_sum(*ora.full_block_ksvd(e)[1:]) if dim == 2
                     else ora.full_block_ksvd_3d(e)["P"])
                assert rel(x[blk], np.linalg.solve(P, b[blk])) <= solve_tol(np.linalg.cond(P)), e
        if dt == 0.0 and dim == 2:
            # sigma_2 of an exactly rank-1 block through the Gram matrix: a rounding-level
            # eigenvalue, so about sqrt(eps) sigma_1 (its factors' product stays at eps level,
            # which the exact apply above shows)
            fs = to_host(ctx.views()["fsig"])
            assert np.all(fs[:, 1] <= 1e-6 * fs[:, 0])
