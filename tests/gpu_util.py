"""Shared helpers for the GPU parity tests (CUDA path vs the CPU oracle)."""
import numpy as np
import torch

import synthetic
from oracle.dg import AdvectionDG, PeriodicMesh

DEV = "cuda:0"


def make_pair(n, nel, dt, vel, max_restart=30, features=0, h=None, mu=None):
    """(CUDA Context, oracle AdvectionDG) for the same problem; mu > n over-integrates."""
    from paper_1704_04549_gb300 import Context
    mesh = PeriodicMesh(nel, h)
    ctx = Context(len(nel), n, nel, mesh.h, dt, vel, max_restart=max_restart,
                  features=features, device=DEV, mu=mu or 0)
    return ctx, AdvectionDG(mesh, n, dt, vel, mu)


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


def solve_tol(kappa, cond_factors=0.0):
    """Tolerance of P^-1 b in FP64 against the oracle's dense LU solve: 1e-12, or
    5 u64 (kappa(P) + cond_factors) where that is larger.  A backward-stable solve,
    the oracle's included, is accurate only to about kappa(P) u64, and the Kronecker
    route multiplies by the explicit inverses of the inverted factor pair (condition
    product cond_factors = cond_1(L_A) cond_1(L_B)), which adds about cond_factors
    u64; no FP64 path can be held closer.  Measured on the GB300, the largest ratio
    of the error to u64 (kappa + cond_factors) over the tests is 2.5 (n = 31 on a
    2 x 2 mesh: kappa 5.3e3, condition product 1.3e4, error 5.0e-12)."""
    return max(FP64_TOL, 5.0 * U64 * (kappa + cond_factors))
