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
