"""Learned Kronecker factors: the MLP and its loss (oracle form).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The network maps an element's input features (the two velocity components at
its n x n nodes and dt / h: 2 n^2 + 1 values) through three hidden layers of
width 512 with the exact GELU, 0.5 x (1 + erf(x / sqrt 2)), to 4 n^2 outputs,
read as vec(A_1), vec(B_1), vec(A_2), vec(B_2) (column-major n x n).  Weights
are stored in BF16 (round to nearest even of the float32 value) and every
product is accumulated in at least FP32; this oracle computes in float64 from
the BF16-rounded weights.

The loss of an element is the gauge-invariant squared relative error of the
rank-2 Kronecker sum on the rearranged block (Sec. 4.1, Eq. NKP):
    L = || A~ / ||A~||_F - sum_k vec(A_k) vec(B_k)^T ||_F^2,
which does not change under (A_k, B_k) -> (c A_k, B_k / c) or a rotation of the
two terms, and whose minimum over the factors is sum_{k > 2} sigma_k^2 /
||A~||_F^2 (Eckart-Young; pinned in tests/test_oracle_mlp.py).  The batch loss is
the mean over elements.  Backward: dL/da_k = -2 R b_k, dL/db_k = -2 R^T a_k with
R the residual matrix, then the chain rule through the layers.

Training uses Adam (``adam_step``, Kingma and Ba 2015, Algorithm 1).

Pinned by central finite differences of the loss with respect to every
parameter of a small network, by the Eckart-Young minimum, by values of the
GELU and its derivative at points where the normal CDF is tabulated, and by
Adam's closed forms (first step, constant gradient) and its convergence on a
quadratic.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

WIDTHS = (513, 512, 512, 512, 1024)     # n = 16


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round float32 values to the nearest BF16 value (ties to even), as float64."""
    x = np.asarray(a, dtype=np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def init_params(seed: int, widths=WIDTHS):
    """Weights W_l [K, N] ~ N(0, 1/K) (float32), biases zero."""
    rng = np.random.Generator(np.random.PCG64(seed))
    params = []
    for K, N in zip(widths[:-1], widths[1:]):
        W = (rng.standard_normal((K, N)) / np.sqrt(K)).astype(np.float32)
        params.append((W, np.zeros(N, dtype=np.float32)))
    return params


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / np.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + erf(x / np.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / np.sqrt(2.0 * np.pi)


def forward(params, X: np.ndarray):
    """Returns the outputs and the pre-activations of every layer."""
    h = np.asarray(X, dtype=np.float64)
    pre = []
    for l, (W, b) in enumerate(params):
        z = h @ bf16_round(W) + np.asarray(b, dtype=np.float64)
        pre.append((h, z))
        h = gelu(z) if l + 1 < len(params) else z
    return h, pre


def backward(params, pre, dout: np.ndarray):
    """Gradients (dW, db) of every layer given dL/d(outputs)."""
    grads = [None] * len(params)
    g = np.asarray(dout, dtype=np.float64)
    for l in range(len(params) - 1, -1, -1):
        h, z = pre[l]
        if l + 1 < len(params):
            g = g * gelu_grad(z)
        W = bf16_round(params[l][0])
        grads[l] = (h.T @ g, g.sum(axis=0))
        g = g @ W.T
    return grads


def adam_step(p, g, m, v, t: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
              eps: float = 1e-8):
    """One Adam update (Kingma and Ba, 2015, Algorithm 1) of parameters p with
    gradient g, first and second moment estimates m, v and step number t >= 1.

    m <- beta1 m + (1 - beta1) g,  v <- beta2 v + (1 - beta2) g^2,
    p <- p - lr (m / (1 - beta1^t)) / (sqrt(v / (1 - beta2^t)) + eps).
    Returns (p, m, v) as float64 arrays."""
    p, g = np.asarray(p, dtype=np.float64), np.asarray(g, dtype=np.float64)
    m = beta1 * np.asarray(m, dtype=np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, dtype=np.float64) + (1.0 - beta2) * g * g
    m_hat = m / (1.0 - beta1 ** t)
    v_hat = v / (1.0 - beta2 ** t)
    return p - lr * m_hat / (np.sqrt(v_hat) + eps), m, v


def unpack(out: np.ndarray, n: int):
    """Rows of outputs -> (A1, B1, A2, B2) as [B, n, n] (column-major vec)."""
    nn = n * n
    mats = []
    for k in range(4):
        v = out[:, k * nn:(k + 1) * nn]
        mats.append(v.reshape(-1, n, n).transpose(0, 2, 1))
    return mats


def factor_loss(At_list, out: np.ndarray, n: int):
    """Mean relative rank-2 error and dL/d(outputs) for rearranged blocks At_list."""
    nn = n * n
    B = out.shape[0]
    loss = 0.0
    dout = np.zeros_like(out, dtype=np.float64)
    for e in range(B):
        At = At_list[e] / np.linalg.norm(At_list[e])
        a1, b1, a2, b2 = (out[e, k * nn:(k + 1) * nn] for k in range(4))
        R = At - np.outer(a1, b1) - np.outer(a2, b2)
        loss += np.sum(R * R)
        dout[e, 0:nn] = -2.0 * R @ b1
        dout[e, nn:2 * nn] = -2.0 * R.T @ a1
        dout[e, 2 * nn:3 * nn] = -2.0 * R @ b2
        dout[e, 3 * nn:4 * nn] = -2.0 * R.T @ a2
    return loss / B, dout / B
