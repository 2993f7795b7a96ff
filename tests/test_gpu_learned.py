"""GPU parity of the learned-factor path (libtpp's factor network) against the
oracle in oracle/mlp.py: network inputs and normalised cores, the forward pass
with BF16 weights, the structured loss and its gradients, the Adam step, and the
learned build with its exact-KSVD fallback inside GMRES."""
import numpy as np
import pytest
import torch

import synthetic
from oracle import mlp
from oracle.ksvd import rearrange
from paper_1704_04549_gb300 import TPP_FEAT_LEARNED, TPP_PC_KRON
from tests.gpu_util import DEV, make_pair, rel, to_dev, to_host

pytestmark = pytest.mark.gpu

DT = 0.05


def _widths(n):
    return (2 * n * n + 1, 512, 512, 512, 4 * n * n)


def _params(n, seed, out_scale=1.0, bias=0.05):
    """Oracle parameters with nonzero biases (so the bias path is exercised)."""
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    ps = mlp.init_params(seed, _widths(n))
    out = []
    for l, (W, b) in enumerate(ps):
        if l == len(ps) - 1:
            W = (W * out_scale).astype(np.float32)
        out.append((W, (bias * rng.standard_normal(b.shape)).astype(np.float32)))
    return out


def _flat(ps):
    return np.concatenate([np.concatenate([W.reshape(-1), b]) for W, b in ps]).astype(np.float32)


def _unflat(flat, n):
    w = _widths(n)
    out, o = [], 0
    for K, N in zip(w[:-1], w[1:]):
        W = flat[o:o + K * N].reshape(K, N)
        o += K * N
        out.append((W, flat[o:o + N]))
        o += N
    return out


def _mesh(n, nel, seed=1712):
    vel = synthetic.fourier_velocity(seed, 2)
    return make_pair(n, nel, DT, vel, features=TPP_FEAT_LEARNED)


@pytest.mark.parametrize("n,nel", [(4, (3, 4)), (7, (2, 3)), (16, (2, 2))])
def test_learned_inputs_match_oracle(n, nel):
    """Features = velocity at the nodes (x fastest) and dt / h; ||A~||_F; the
    normalised core has the singular values of A~ / ||A~||_F (A~ = Q M Q^T)."""
    ctx, dg = _mesh(n, nel)
    X, Mn, norms = ctx.tpp_learned_inputs()
    X, Mn, norms = to_host(X), to_host(Mn), to_host(norms)
    r, nn = ctx.tpp_core_size(), n * n
    assert r == n + min(nn - n, n + 2)
    assert X.shape[0] == dg.mesh.num_elem
    for e in range(dg.mesh.num_elem):
        a = dg.velocity_at(dg.volume_points(e))
        assert np.max(np.abs(X[e, :nn] - a[:, 0])) <= 1e-6 * max(1.0, np.abs(a).max())
        assert np.max(np.abs(X[e, nn:2 * nn] - a[:, 1])) <= 1e-6 * max(1.0, np.abs(a).max())
        assert X[e, 2 * nn] == np.float32(DT / dg.mesh.h)
        At = rearrange(dg.element_block(e), n, n, n, n)
        assert abs(norms[e] - np.linalg.norm(At)) <= 1e-13 * np.linalg.norm(At)
        s_ref = np.linalg.svd(At / np.linalg.norm(At), compute_uv=False)
        s = np.linalg.svd(Mn[e].reshape(r, r, order="F"), compute_uv=False)
        assert np.max(np.abs(s - s_ref[:r])) <= 1e-13
        assert np.all(s_ref[r:] <= 1e-13)       # A~ has rank <= r


@pytest.mark.parametrize("n,B", [(4, 1), (4, 70), (5, 129), (16, 33)])
def test_forward_matches_oracle(n, B):
    """FP32 accumulation over at most 513 BF16-weighted terms per layer, four
    layers: norm-wise relative error well below 1e-4."""
    from paper_1704_04549_gb300 import Mlp
    ps = _params(n, 11)
    net = Mlp(n, max_batch=max(B, 8), params=_flat(ps))
    rng = np.random.Generator(np.random.PCG64(12))
    X = rng.uniform(-1.5, 1.5, (B, _widths(n)[0])).astype(np.float32)
    out = to_host(net.forward(torch.as_tensor(X, device=DEV)))
    ref, _ = mlp.forward(ps, X.astype(np.float64))
    assert rel(out, ref) <= 1e-4
    # every row (tile edges and the ragged tail included)
    for i in range(B):
        assert rel(out[i], ref[i]) <= 1e-4, i
    assert np.array_equal(net.get_params(), _flat(ps))


@pytest.mark.parametrize("n,nel", [(4, (5, 6)), (6, (3, 3))])
def test_loss_and_gradients_match_oracle(n, nel):
    """The structured loss (through the core M) equals the dense loss on A~; the
    gradients of every layer match the oracle's back-propagation."""
    from paper_1704_04549_gb300 import Mlp
    ctx, dg = _mesh(n, nel)
    X, Mn, _ = ctx.tpp_learned_inputs()
    E = X.shape[0]
    ps = _params(n, 21, out_scale=0.2)
    net = Mlp(n, max_batch=64, params=_flat(ps))
    loss = float(to_host(net.train_step(ctx, X, Mn, lr=0.0))[0])
    g = to_host(net.gradients())
    Xh = to_host(X).astype(np.float64)
    out, pre = mlp.forward(ps, Xh)
    At = [rearrange(dg.element_block(e), n, n, n, n) for e in range(E)]
    ref_loss, dout = mlp.factor_loss(At, out, n)
    assert abs(loss - ref_loss) <= 1e-4 * max(1.0, ref_loss)
    grads = mlp.backward(ps, pre, dout)
    gg = _unflat(g, n)
    for l, ((dW, db), (gW, gb)) in enumerate(zip(grads, gg)):
        assert rel(gW, dW) <= 1e-3, (l, rel(gW, dW))
        assert rel(gb, db) <= 1e-3, (l, rel(gb, db))
    # the parameters are untouched by an lr = 0 step
    assert np.array_equal(net.get_params(), _flat(ps))


def test_loss_is_gauge_invariant():
    """(A_k, B_k) -> (c A_k, B_k / c) and a swap of the two terms leave the GPU
    loss unchanged (outputs fed through a network whose last layer realises the
    transformation exactly: weights scaled by powers of two, columns permuted)."""
    from paper_1704_04549_gb300 import Mlp
    n = 4
    nn = n * n
    ctx, _ = _mesh(n, (3, 3))
    X, Mn, _ = ctx.tpp_learned_inputs()
    ps = _params(n, 31, out_scale=0.2)
    W3, b3 = ps[3]
    W3s, b3s = W3.copy(), b3.copy()
    for k, c in ((0, 2.0), (1, 0.5), (2, 0.25), (3, 4.0)):   # a1*2, b1/2, a2/4, b2*4
        W3s[:, k * nn:(k + 1) * nn] *= c
        b3s[k * nn:(k + 1) * nn] *= c
    ps2 = ps[:3] + [(W3s, b3s)]
    net = Mlp(n, max_batch=16, params=_flat(ps))
    l1 = float(to_host(net.train_step(ctx, X, Mn, lr=0.0))[0])
    net.set_params(_flat(ps2))
    l2 = float(to_host(net.train_step(ctx, X, Mn, lr=0.0))[0])
    perm = np.concatenate([np.arange(2 * nn, 4 * nn), np.arange(0, 2 * nn)])
    net.set_params(_flat(ps[:3] + [(W3[:, perm].copy(), b3[perm].copy())]))
    l3 = float(to_host(net.train_step(ctx, X, Mn, lr=0.0))[0])
    assert abs(l1 - l2) <= 1e-6 * max(1.0, l1)
    assert abs(l1 - l3) <= 1e-6 * max(1.0, l1)


def test_adam_steps_match_oracle():
    """Three Adam steps against the oracle's update (Kingma and Ba, Algorithm 1) fed
    with the GPU's gradients of each step: FP32 moments and parameters, so the
    parameters agree to FP32 rounding of updates of size lr."""
    from paper_1704_04549_gb300 import Mlp
    n = 4
    ctx, _ = _mesh(n, (3, 3))
    X, Mn, _ = ctx.tpp_learned_inputs()
    ps = _params(n, 41, out_scale=0.2)
    p = _flat(ps).astype(np.float64)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    net = Mlp(n, max_batch=16, params=_flat(ps))
    for t in range(1, 4):
        net.train_step(ctx, X, Mn, lr=1e-3)
        g = to_host(net.gradients()).astype(np.float64)
        p, m, v = mlp.adam_step(p, g, m, v, t, 1e-3)
        p1 = net.get_params().astype(np.float64)
        assert np.max(np.abs(p1 - p)) <= 2e-6, t
        p = p1                 # continue from the GPU's parameters (FP32 state)


def test_training_reduces_loss():
    from paper_1704_04549_gb300 import Mlp
    n = 4
    ctx, _ = _mesh(n, (16, 16))
    X, Mn, _ = ctx.tpp_learned_inputs()
    net = Mlp(n, max_batch=64, params=_flat(_params(n, 51, out_scale=0.1, bias=0.0)))
    first = float(to_host(net.train_step(ctx, X[:64], Mn[:64], lr=0.0))[0])
    for it in range(400):
        s = (it % 4) * 64
        net.train_step(ctx, X[s:s + 64], Mn[s:s + 64], lr=2e-4)
    last = float(to_host(net.train_step(ctx, X[:64], Mn[:64], lr=0.0))[0])
    assert last <= 0.1 * first, (first, last)


def _elem_errors(ctx, dg, net, n):
    X, _, norms = ctx.tpp_learned_inputs()
    mb = net.max_batch
    out = np.concatenate([to_host(net.forward(X[s:s + mb])) for s in range(0, X.shape[0], mb)])
    out = out.astype(np.float64)
    nn, errs, Ps = n * n, [], []
    for e in range(X.shape[0]):
        At = rearrange(dg.element_block(e), n, n, n, n)
        a1, b1, a2, b2 = (out[e, k * nn:(k + 1) * nn] for k in range(4))
        R = At / np.linalg.norm(At) - np.outer(a1, b1) - np.outer(a2, b2)
        errs.append(np.linalg.norm(R))
        A = [v.reshape(n, n, order="F") for v in (a1, b1, a2, b2)]
        Ps.append(np.linalg.norm(At) * (np.kron(A[0], A[1]) + np.kron(A[2], A[3])))
    return np.array(errs), Ps


def test_learned_build_accepts_and_falls_back():
    """threshold 0: every element takes the exact KSVD (bit-identical to
    tpp_build_factors); threshold inf: every element keeps the network's factors,
    P = ||A~|| (a1 (x) b1 + a2 (x) b2); in between, the fallback count is the number
    of elements whose relative rank-2 error exceeds the threshold."""
    from paper_1704_04549_gb300 import Mlp
    n = 4
    ctx, dg = _mesh(n, (4, 5))
    ref_ctx, _ = _mesh(n, (4, 5))
    ref_ctx.tpp_build_factors()
    net = Mlp(n, max_batch=8, params=_flat(_params(n, 61, out_scale=0.1)))
    E = ctx.num_elem
    errs, Ps = _elem_errors(ctx, dg, net, n)
    rep = ctx.tpp_build_factors_learned(net, threshold=0.0)
    assert rep["num_fallback"] == E
    v, vr = ctx.views(), ref_ctx.views()
    for k in ("sigma", "A1", "B1", "A2", "B2", "SA", "SB", "Q1", "T1", "cond"):
        if v[k] is not None:
            assert torch.equal(v[k], vr[k]), k
    rep = ctx.tpp_build_factors_learned(net, threshold=np.inf)
    assert rep["num_fallback"] == 0
    v = ctx.views()
    A1, B1, A2, B2 = (to_host(v[k]) for k in ("A1", "B1", "A2", "B2"))
    for e in range(E):
        P = np.kron(A1[e], B1[e]) + np.kron(A2[e], B2[e])   # gauge shift leaves P unchanged
        assert rel(P, Ps[e]) <= 1e-6, e                     # FP32 outputs
    thr = float(np.median(errs))
    rep = ctx.tpp_build_factors_learned(net, threshold=thr)
    margin = np.abs(errs - thr) > 1e-6 * thr
    expect = int(np.sum(errs[margin] > thr))
    assert expect <= rep["num_fallback"] <= expect + int(np.sum(~margin))


def test_learned_factors_in_gmres():
    """A briefly trained network on a 16 x 16 mesh: the learned build with the
    0.05 fallback threshold gives a preconditioner with which GMRES reaches the
    1e-8 true residual, in at most twice the iterations of the exact KSVD (+ 2)."""
    from paper_1704_04549_gb300 import Mlp
    n = 4
    ctx, dg = _mesh(n, (16, 16))
    X, Mn, _ = ctx.tpp_learned_inputs()
    net = Mlp(n, max_batch=64, params=_flat(_params(n, 71, out_scale=0.1, bias=0.0)))
    for it in range(600):
        s = (it % 4) * 64
        net.train_step(ctx, X[s:s + 64], Mn[s:s + 64], lr=2e-4 if it < 400 else 5e-5)
    b = synthetic.rhs(1713, dg.ndof)
    ctx.tpp_build_factors()
    _, r_exact = ctx.gmres_solve(to_dev(b), pc=TPP_PC_KRON, rtol=1e-8)
    rep = ctx.tpp_build_factors_learned(net, threshold=0.05)
    x, r = ctx.gmres_solve(to_dev(b), pc=TPP_PC_KRON, rtol=1e-8)
    assert r["converged"] and r["true_rel_res"] <= 1e-8
    assert r["iters"] <= 2 * r_exact["iters"] + 2, (r["iters"], r_exact["iters"], rep)
    Ax = to_host(ctx.dg_apply_sumfact(x))
    assert np.linalg.norm(Ax - b) <= 1.0001e-8 * np.linalg.norm(b)


def test_solve_learned_iteration_fallback():
    """tpp_solve_learned's second fallback: with every element on an untrained
    network's factors (threshold infinity) the first GMRES solve exceeds its
    iteration limit, every element is rebuilt by the exact KSVD and GMRES continues
    from the current iterate to the 1e-8 true residual (checked with the oracle's
    S); both solves together stay within max_iters."""
    from paper_1704_04549_gb300 import Mlp
    n = 4
    ctx, dg = _mesh(n, (6, 6))
    net = Mlp(n, max_batch=64, params=_flat(_params(n, 81, out_scale=0.1)))
    b = synthetic.rhs(1714, dg.ndof)
    S = dg.global_matrix()
    ctx.tpp_build_factors()
    _, r_exact = ctx.gmres_solve(to_dev(b), pc=TPP_PC_KRON, rtol=1e-8)
    limit = 3
    x, r = ctx.tpp_solve_learned(net, to_dev(b), threshold=np.inf, iter_limit=limit, rtol=1e-8)
    assert r["rebuilt"] == 1 and r["build"]["num_fallback"] == dg.mesh.num_elem
    assert r["converged"] and r["true_rel_res"] <= 1e-8
    assert limit < r["iters"] <= limit + r_exact["iters"] + 2
    xh = to_host(x)
    assert np.linalg.norm(b - S @ xh) <= 1.0001e-8 * np.linalg.norm(b)
    # the caller's max_iters bounds both solves: 3 + 2 steps are not enough
    x, r = ctx.tpp_solve_learned(net, to_dev(b), threshold=np.inf, iter_limit=limit,
                                 rtol=1e-8, max_iters=limit + 2, check=False)
    assert r["rebuilt"] == 1 and not r["converged"] and r["iters"] == limit + 2
    assert r["status"] == 4
    # threshold 0: every element takes the exact KSVD, the first solve converges
    # within its limit and nothing is rebuilt
    x, r = ctx.tpp_solve_learned(net, to_dev(b), threshold=0.0, iter_limit=r_exact["iters"] + 1,
                                 rtol=1e-8)
    assert r["rebuilt"] == 0 and r["converged"] and r["iters"] == r_exact["iters"]


def _build_ms(fn, reps=5):
    """Median device time (ms) of fn() on the current stream."""
    times = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    return float(np.median(times))


def test_trained_network_gain_on_the_mesh():
    """What the trained network gains over the exact construction on the 64 x 64 mesh
    (n = 16, unit quads, dt = 0.05, field 1705, which training never sees): trained
    on 20,000 isolated elements of ten other fields (30 epochs), it keeps its own
    factors on most elements at the 5% error threshold, GMRES with the learned
    preconditioner reaches the 1e-8 true residual (checked with the oracle's
    sum-factorised matvec) in at most the exact preconditioner's iterations + 2, and
    the learned build (network, error check, exact KSVD of the fallback elements,
    inverses and Schur forms) takes less time than the exact build."""
    from paper_1704_04549_gb300 import learned as LN
    n = 16
    Xt, Mt, _, basis = LN.element_samples(n, 20000, range(1801, 1811), seed=1800)
    net = LN.Mlp(n, max_batch=4096, params=LN.default_params(n, 1800))
    hist = LN.train(net, basis, Xt, Mt, 30, batch=512, lr=1e-3, lr_min=1e-5)
    ctx, dg = make_pair(n, (64, 64), 0.05, synthetic.fourier_velocity(1705, 2),
                        features=TPP_FEAT_LEARNED, h=1.0)
    b = synthetic.rhs(1706, dg.ndof)
    E = dg.mesh.num_elem
    ctx.tpp_build_factors()
    t_exact = _build_ms(ctx.tpp_build_factors)
    _, r_exact = ctx.gmres_solve(to_dev(b), pc=TPP_PC_KRON, rtol=1e-8)
    t_learned = _build_ms(lambda: ctx.tpp_build_factors_learned(net, 0.05))
    rep = ctx.tpp_build_factors_learned(net, 0.05)
    x, r = ctx.gmres_solve(to_dev(b), pc=TPP_PC_KRON, rtol=1e-8)
    print(f"learned gain, 64x64 n=16: training loss {hist[0]:.3e} -> {hist[-1]:.3e}; "
          f"{E - rep['num_fallback']} of {E} elements keep the network's factors; "
          f"build {t_exact:.2f} ms exact -> {t_learned:.2f} ms learned; GMRES "
          f"{r_exact['iters']} -> {r['iters']} iterations")
    assert hist[-1] < 0.2 * hist[0]
    assert rep["num_fallback"] <= E // 2
    assert r["converged"] and r["iters"] <= r_exact["iters"] + 2
    Ax = dg.apply_sumfact(to_host(x))
    assert np.linalg.norm(Ax - b) <= 1.0001e-8 * np.linalg.norm(b)
    assert t_learned < t_exact


@pytest.mark.parametrize("n,B", [(16, 300)])
def test_large_batch_gradients_match_oracle(n, B):
    """A batch of three 128-row tiles with a ragged tail at n = 16 (output width 1024,
    input width 513): loss and every layer's gradients against the oracle."""
    from paper_1704_04549_gb300 import Mlp
    ctx, dg = _mesh(n, (10, 30))
    X, Mn, _ = ctx.tpp_learned_inputs()
    assert X.shape[0] == B
    ps = _params(n, 23, out_scale=0.2)
    net = Mlp(n, max_batch=512, params=_flat(ps))
    loss = float(to_host(net.train_step(ctx, X, Mn, lr=0.0))[0])
    g = to_host(net.gradients())
    out, pre = mlp.forward(ps, to_host(X).astype(np.float64))
    At = [rearrange(dg.element_block(e), n, n, n, n) for e in range(B)]
    ref_loss, dout = mlp.factor_loss(At, out, n)
    assert abs(loss - ref_loss) <= 1e-4 * max(1.0, ref_loss)
    for l, ((dW, db), (gW, gb)) in enumerate(zip(mlp.backward(ps, pre, dout), _unflat(g, n))):
        assert rel(gW, dW) <= 1e-3, (l, rel(gW, dW))
        assert rel(gb, db) <= 1e-3, (l, rel(gb, db))
