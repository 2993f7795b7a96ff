"""Shared helpers for the GPU parity tests (CUDA path vs the CPU oracle)."""
import numpy as np
import torch

import synthetic
from oracle.dg import AdvectionDG, PeriodicMesh

DEV = "cuda:0"


def make_pair(n, nel, dt, vel, max_restart=30, features=0, h=None):
    """(CUDA Context, oracle AdvectionDG) for the same problem."""
    from paper_1704_04549_gb300 import Context
    mesh = PeriodicMesh(nel, h)
    ctx = Context(len(nel), n, nel, mesh.h, dt, vel, max_restart=max_restart,
                  features=features, device=DEV)
    return ctx, AdvectionDG(mesh, n, dt, vel)


def to_dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


def to_host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


# Stated relative tolerance of every FP64 result against the oracle (operator, P,
# sigma_k, P^-1 b element by element).
FP64_TOL = 1e-12
U64 = 2.0 ** -53


def solve_tol(kappa):
    """Tolerance of an FP64 solve with a matrix of condition number kappa against the
    oracle's LU solve: 1e-12, or 5 kappa u64 where that is larger.  A backward-stable
    solve (the oracle's included) is only accurate to about kappa u64, so no FP64
    method can be held closer; measured on the GB300, the largest ratio of the error
    to kappa u64 over the tests is 2.1 (n = 31, kappa(P) = 1.8e4: 4.1e-12)."""
    return max(FP64_TOL, 5.0 * kappa * U64)
