"""Thin binding of libtpp's factor network (tpp_mlp_*): an MLP that maps an
element's velocity samples to its rank-2 Kronecker factors.  Marshalling only;
the forward pass, the loss, back-propagation and Adam run in libtpp's kernels.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib as L
from .solver import _ptr, _stream


class Mlp:
    """A tpp_mlp of order n with its workspace (batches of at most max_batch)."""

    def __init__(self, n: int, max_batch: int = 4096, params=None, device: str = "cuda:0",
                 stream=None):
        if not torch.cuda.is_available():
            raise RuntimeError("libtpp needs a CUDA device; there is no CPU path")
        self.lib = L.load()
        self.device = torch.device(device)
        self.n, self.max_batch = int(n), int(max_batch)
        self.num_params = int(self.lib.tpp_mlp_num_params(self.n))
        nbytes = self.lib.tpp_mlp_workspace_bytes(self.n, self.max_batch)
        if self.num_params < 0 or nbytes == 0:
            raise L.TppError(1, "tpp_mlp_workspace_bytes")
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        ptr = (self.workspace.data_ptr() + 255) & ~255
        net = C.c_void_p()
        with torch.cuda.device(self.device):
            L.check(self.lib.tpp_mlp_create(C.byref(net), self.n, self.max_batch, C.c_void_p(ptr),
                                            nbytes, _stream(stream)), "tpp_mlp_create")
        self._net = net
        self._loss = torch.zeros(1, dtype=torch.float32, device=self.device)
        if params is not None:
            self.set_params(params, stream)

    def __del__(self):
        net = getattr(self, "_net", None)
        if net is not None and net.value:
            self.lib.tpp_mlp_destroy(net)
            self._net = None

    @property
    def widths(self):
        return (2 * self.n * self.n + 1, 512, 512, 512, 4 * self.n * self.n)

    def set_params(self, params, stream=None):
        """params: flat FP32 array (W_l [K][N] row-major then b_l, l = 0..3)."""
        host = np.ascontiguousarray(params, dtype=np.float32).reshape(-1)
        if host.size != self.num_params:
            raise ValueError(f"expected {self.num_params} parameters, got {host.size}")
        self._host = host                  # kept alive for the asynchronous copy
        L.check(self.lib.tpp_mlp_set_params(self._net, host.ctypes.data_as(C.c_void_p),
                                            _stream(stream)), "tpp_mlp_set_params")
        torch.cuda.current_stream(self.device).synchronize() if stream is None \
            else stream.synchronize()

    def get_params(self, stream=None) -> np.ndarray:
        host = np.empty(self.num_params, dtype=np.float32)
        L.check(self.lib.tpp_mlp_get_params(self._net, host.ctypes.data_as(C.c_void_p),
                                            _stream(stream)), "tpp_mlp_get_params")
        return host

    def _batch(self, X):
        if not (isinstance(X, torch.Tensor) and X.is_cuda and X.dtype == torch.float32
                and X.is_contiguous() and X.dim() == 2 and X.shape[1] == self.widths[0]
                and 1 <= X.shape[0] <= self.max_batch):
            raise ValueError("X must be a contiguous float32 CUDA tensor [B, 2n^2+1], "
                             f"1 <= B <= {self.max_batch}")
        return X

    def forward(self, X, stream=None):
        X = self._batch(X)
        out = torch.empty((X.shape[0], self.widths[4]), dtype=torch.float32, device=self.device)
        L.check(self.lib.tpp_mlp_forward(self._net, _ptr(X), X.shape[0], _ptr(out),
                                         _stream(stream)), "tpp_mlp_forward")
        return out

    def train_step(self, basis, X, Mn, lr: float, stream=None):
        """Loss (device float tensor [1], the batch mean) of one batch; with lr > 0 one
        Adam step.  basis: a 2D Context of the same n (its structure basis)."""
        X = self._batch(X)
        if not (Mn.is_cuda and Mn.dtype == torch.float64 and Mn.is_contiguous()
                and Mn.shape[0] == X.shape[0]):
            raise ValueError("Mn must be a contiguous float64 CUDA tensor [B, r*r]")
        L.check(self.lib.tpp_mlp_train_step(self._net, basis._ctx, _ptr(X), _ptr(Mn), X.shape[0],
                                            float(lr), _ptr(self._loss), _stream(stream)),
                "tpp_mlp_train_step")
        return self._loss

    def element_loss(self, basis, X, Mn, stream=None) -> torch.Tensor:
        """Per-element loss L_e (float64 [B]) of the network's factors."""
        X = self._batch(X)
        out = torch.empty(X.shape[0], dtype=torch.float64, device=self.device)
        L.check(self.lib.tpp_mlp_element_loss(self._net, basis._ctx, _ptr(X), _ptr(Mn), X.shape[0],
                                              _ptr(out), _stream(stream)), "tpp_mlp_element_loss")
        return out

    def gradients(self) -> torch.Tensor:
        """Copy of the gradients of the last train step (parameter layout)."""
        addr = self.lib.tpp_mlp_gradients(self._net)
        out = torch.empty(self.num_params, dtype=torch.float32, device=self.device)
        L.check(self.lib.tpp_copy_device(_ptr(out), C.c_void_p(addr), out.numel() * 4,
                                         _stream(None)), "tpp_copy_device")
        return out


# -- training utilities (host orchestration of the calls above) ------------------

def default_params(n: int, seed: int, out_scale: float = 0.1) -> np.ndarray:
    """Initial parameters: W_l ~ N(0, 1/K_l) (the output layer scaled by out_scale,
    so that the first factors are small), zero biases; flat FP32 layout."""
    rng = np.random.Generator(np.random.PCG64(seed))
    w = (2 * n * n + 1, 512, 512, 512, 4 * n * n)
    parts = []
    for l, (K, N) in enumerate(zip(w[:-1], w[1:])):
        W = rng.standard_normal((K, N)) / np.sqrt(K)
        if l == 3:
            W *= out_scale
        parts += [W.reshape(-1), np.zeros(N)]
    return np.concatenate(parts).astype(np.float32)


def element_samples(n: int, count: int, field_seeds, *, h: float = 1.0, span: float = 1.0 / 64,
                    dt: float = 0.05, seed: int = 0, device: str = "cuda:0"):
    """Network inputs X [count, 2n^2+1], normalised cores Mn [count, r^2] and block
    norms of `count` isolated elements drawn evenly from random-Fourier velocity
    fields (one per seed in field_seeds), centres uniform in the unit square, width h,
    field sampled over `span`; rows interleaved in a seeded random order.  Returns
    (X, Mn, norms, basis) with basis a small context of the same n (structure basis)."""
    import synthetic
    from .solver import Context
    seeds = list(field_seeds)
    rng = np.random.Generator(np.random.PCG64(seed))
    per = [count // len(seeds) + (1 if i < count % len(seeds) else 0) for i in range(len(seeds))]
    Xs, Ms, Ns = [], [], []
    for fs, E in zip(seeds, per):
        if E == 0:
            continue
        ctx = Context(2, n, (E,), h, dt, synthetic.fourier_velocity(fs, 2), max_restart=1,
                      device=device, batch_rhs=1, centres=rng.random((E, 2)), batch_span=span)
        X, Mn, nr = ctx.tpp_learned_inputs()
        Xs.append(X)
        Ms.append(Mn)
        Ns.append(nr)
        del ctx
    order = torch.as_tensor(rng.permutation(count), device=device)
    X = torch.cat(Xs).index_select(0, order).contiguous()
    Mn = torch.cat(Ms).index_select(0, order).contiguous()
    nr = torch.cat(Ns).index_select(0, order).contiguous()
    basis = Context(2, n, (1,), h, dt, synthetic.fourier_velocity(seeds[0], 2), max_restart=1,
                    device=device, batch_rhs=1, centres=np.full((1, 2), 0.5), batch_span=span)
    return X, Mn, nr, basis


def train(net: Mlp, basis, X, Mn, epochs: int, batch: int = 512, lr: float = 1e-3,
          lr_min: float = 1e-5, stream=None):
    """Adam over contiguous minibatches (the rows are pre-shuffled), cosine learning
    rate from lr to lr_min.  Returns the mean training loss of every epoch."""
    E = X.shape[0]
    nb = (E + batch - 1) // batch
    total = epochs * nb
    hist = []
    acc = torch.zeros(1, dtype=torch.float32, device=net.device)
    step = 0
    for ep in range(epochs):
        acc.zero_()
        for i in range(nb):
            s0, s1 = i * batch, min(E, (i + 1) * batch)
            rate = lr_min + 0.5 * (lr - lr_min) * (1.0 + np.cos(np.pi * step / max(1, total - 1)))
            acc += net.train_step(basis, X[s0:s1], Mn[s0:s1], rate, stream)
            step += 1
        hist.append(acc)
        acc = torch.zeros(1, dtype=torch.float32, device=net.device)
    return [float(h.item()) / nb for h in hist]


def element_errors(net: Mlp, basis, X, Mn, stream=None) -> torch.Tensor:
    """Relative rank-2 error sqrt(L_e) of the network's factors, every element."""
    mb = net.max_batch
    parts = [net.element_loss(basis, X[s:s + mb], Mn[s:s + mb], stream)
             for s in range(0, X.shape[0], mb)]
    return torch.cat(parts).clamp_min(0.0).sqrt()
