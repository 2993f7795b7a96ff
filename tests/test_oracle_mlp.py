"""Pins of the learned-factor oracle: finite differences and Eckart-Young."""
import numpy as np

import synthetic
from oracle import mlp
from oracle.dg import IsolatedElements
from oracle.ksvd import ksvd_2d, rearrange


def _blocks(n, count, seed=3):
    rng = np.random.Generator(np.random.PCG64(seed))
    iso = IsolatedElements(n, 1.0, rng.random((count, 2)), 0.05,
                           synthetic.fourier_velocity(21, 2), span=1.0 / 64)
    return [rearrange(iso.block(e), n, n, n, n) for e in range(count)], iso


def test_bf16_rounding():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -3.14159, 65504.0], dtype=np.float32)
    r = mlp.bf16_round(x)
    # exactly representable values stay; others move by at most half a BF16 ulp (2^-8 relative)
    assert np.all(np.abs(r - x) <= 2.0 ** -8 * np.abs(x))
    assert mlp.bf16_round(np.float32(1.0 + 2 ** -7))[()] == 1.0 + 2 ** -7
    # ties go to even: 1 + 2^-8 lies halfway between 1 and 1 + 2^-7
    assert mlp.bf16_round(np.float32(1.0 + 2 ** -8))[()] == 1.0


def test_eckart_young_minimum():
    """At the exact top-2 Kronecker factors the loss is sum_{k>2} sigma_k^2 / ||A~||^2."""
    n = 4
    At, iso = _blocks(n, 3)
    out = []
    for e in range(3):
        s, As, Bs = ksvd_2d(iso.block(e), n, r=2)
        nrm = np.linalg.norm(At[e])
        row = [As[0].reshape(-1, order="F") / np.sqrt(nrm), Bs[0].reshape(-1, order="F") / np.sqrt(nrm),
               As[1].reshape(-1, order="F") / np.sqrt(nrm), Bs[1].reshape(-1, order="F") / np.sqrt(nrm)]
        out.append(np.concatenate(row))
    loss, _ = mlp.factor_loss(At, np.array(out), n)
    ref = np.mean([np.sum(np.linalg.svd(A, compute_uv=False)[2:] ** 2) / np.sum(A * A) for A in At])
    assert abs(loss - ref) <= 1e-12


def test_loss_gradient_finite_differences():
    n = 3
    At, _ = _blocks(n, 2, seed=5)
    rng = np.random.Generator(np.random.PCG64(7))
    out = rng.standard_normal((2, 4 * n * n)) * 0.3
    loss, dout = mlp.factor_loss(At, out, n)
    eps = 1e-6
    for idx in [(0, 0), (0, 10), (1, 20), (1, 35)]:
        o1, o2 = out.copy(), out.copy()
        o1[idx] += eps
        o2[idx] -= eps
        fd = (mlp.factor_loss(At, o1, n)[0] - mlp.factor_loss(At, o2, n)[0]) / (2 * eps)
        assert abs(fd - dout[idx]) <= 1e-7 * max(1.0, abs(fd))


def test_network_gradient_finite_differences():
    """Every parameter of a small network against central differences of the loss
    (weights entering through their BF16 rounding: differences are taken in the
    rounded weights, which the backward pass uses)."""
    n = 2
    widths = (2 * n * n + 1, 6, 5, 4, 4 * n * n)
    params = mlp.init_params(3, widths)
    params = [(mlp.bf16_round(W).astype(np.float32), (np.arange(len(b)) * 0.01).astype(np.float32))
              for W, b in params]
    At, _ = _blocks(n, 3, seed=9)
    rng = np.random.Generator(np.random.PCG64(4))
    X = rng.standard_normal((3, widths[0]))

    def loss_of(ps):
        out, _ = mlp.forward(ps, X)
        return mlp.factor_loss(At, out, n)[0]

    out, pre = mlp.forward(params, X)
    _, dout = mlp.factor_loss(At, out, n)
    grads = mlp.backward(params, pre, dout)
    P64 = [(W.astype(np.float64), b.astype(np.float64)) for W, b in params]

    def loss64(ps):       # same network in float64 weights (already BF16 values)
        h = X
        for l, (W, b) in enumerate(ps):
            z = h @ W + b
            h = mlp.gelu(z) if l + 1 < len(ps) else z
        return mlp.factor_loss(At, h, n)[0]

    eps = 1e-6
    for l in range(4):
        W, b = P64[l]
        for (i, j) in [(0, 0), (W.shape[0] - 1, W.shape[1] - 1), (1, 2 % W.shape[1])]:
            Wp, Wm = W.copy(), W.copy()
            Wp[i, j] += eps
            Wm[i, j] -= eps
            ps_p = P64[:l] + [(Wp, b)] + P64[l + 1:]
            ps_m = P64[:l] + [(Wm, b)] + P64[l + 1:]
            fd = (loss64(ps_p) - loss64(ps_m)) / (2 * eps)
            assert abs(fd - grads[l][0][i, j]) <= 1e-6 * max(1.0, abs(fd))
        bp, bm = b.copy(), b.copy()
        bp[0] += eps
        bm[0] -= eps
        fd = (loss64(P64[:l] + [(W, bp)] + P64[l + 1:]) - loss64(P64[:l] + [(W, bm)] + P64[l + 1:])) / (2 * eps)
        assert abs(fd - grads[l][1][0]) <= 1e-6 * max(1.0, abs(fd))
    assert abs(loss_of(params) - loss64(P64)) <= 1e-12


def test_gelu_known_values():
    """GELU(x) = x Phi(x) with the standard normal CDF: Phi(1) = 0.8413447460685429,
    phi(1) = exp(-1/2) / sqrt(2 pi) = 0.24197072451914337 (tabulated values).
    The tanh approximation misses GELU(1) by 2e-4, so it would fail here."""
    x = np.array([0.0, 1.0, -1.0, 2.0, -3.0])
    g = mlp.gelu(x)
    assert g[0] == 0.0
    assert abs(g[1] - 0.8413447460685429) <= 1e-15
    assert abs(g[2] + 0.15865525393145707) <= 1e-15
    assert abs(g[3] - 2.0 * 0.9772498680518208) <= 1e-15       # Phi(2)
    assert abs(g[4] + 3.0 * 0.0013498980316300946) <= 1e-15    # Phi(-3)
    # GELU(x) - GELU(-x) = x (Phi(x) + Phi(-x) = 1)
    xs = np.linspace(-5.0, 5.0, 41)
    assert np.max(np.abs(mlp.gelu(xs) - mlp.gelu(-xs) - xs)) <= 1e-14
    # derivative: Phi(x) + x phi(x)
    d = mlp.gelu_grad(np.array([0.0, 1.0, -1.0]))
    assert d[0] == 0.5
    assert abs(d[1] - (0.8413447460685429 + 0.24197072451914337)) <= 1e-15
    assert abs(d[2] - (0.15865525393145707 - 0.24197072451914337)) <= 1e-15


def test_adam_closed_forms():
    """Step 1: the bias corrections make m_hat = g and v_hat = g^2, so the move is
    lr g / (|g| + eps).  A constant gradient keeps m_hat = g, v_hat = g^2 at every
    step (the purpose of the bias correction)."""
    rng = np.random.Generator(np.random.PCG64(17))
    g = rng.standard_normal(50) * np.logspace(-6, 2, 50)
    p0 = rng.standard_normal(50)
    z = np.zeros(50)
    p1, m, v = mlp.adam_step(p0, g, z, z, 1, 1e-3)
    assert np.max(np.abs(p1 - (p0 - 1e-3 * g / (np.abs(g) + 1e-8)))) <= 1e-15
    p, m, v = p0, z, z
    for t in range(1, 41):
        p_prev = p
        p, m, v = mlp.adam_step(p, g, m, v, t, 1e-2)
        step = p_prev - p
        assert np.max(np.abs(step - 1e-2 * g / (np.abs(g) + 1e-8)) / 1e-2) <= 1e-12


def test_adam_minimises_a_quadratic():
    """f(p) = sum (p - c)^2 from p = 0: Adam with lr 0.05 ends within 1e-2 of c."""
    c = np.array([3.0, -1.0, 0.25, 10.0])
    p, m, v = np.zeros(4), np.zeros(4), np.zeros(4)
    for t in range(1, 3001):
        p, m, v = mlp.adam_step(p, 2.0 * (p - c), m, v, t, 0.05 if t < 2000 else 0.005)
    assert np.max(np.abs(p - c)) <= 1e-2
