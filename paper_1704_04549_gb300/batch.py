"""Mixed-degree batches of block-diagonal DG advection systems.

Each element of the batch is isolated (its system is its own diagonal block:
mass, volume and outflow face terms, no neighbour coupling) and carries R
right-hand sides.  Elements are grouped by (dimension, n); each group is one
libtpp context in batch mode, so every kernel of a group runs with one degree
and the factor build, the Kronecker apply and the Krylov solve treat all the
group's systems at once.  Groups run one after another on the caller's stream.
This module only sequences calls to the C ABI (through Context).
"""
from __future__ import annotations

import numpy as np
import torch

import synthetic
from . import _lib as L


def solve_group(group, rhs: int, h: float, dt: float, velocity, *, span: float = 0.0,
                inner_iters: int = 0, rtol: float = 1e-8, max_iters: int = 3000,
                restart: int = 30, device: str = "cuda:0", steps: int = 1, warmup: int = 0,
                use_graph: bool = False):
    """Build the factors of one degree group and solve its systems; returns a dict
    with the device times (CUDA events) of the timed steps and the solve report."""
    from .solver import Context
    ctx = Context(group.dim, group.n, (len(group.ids),), h, dt, velocity,
                  max_restart=restart, features=L.TPP_FEAT_MIXED, device=device,
                  batch_rhs=rhs, centres=group.centres, batch_span=span)
    b = torch.as_tensor(synthetic.rhs(group.rhs_seed, ctx.num_dofs), device=device)
    x = torch.zeros_like(b)
    kw = dict(restart=restart, rtol=rtol, max_iters=max_iters, pc=L.TPP_PC_KRON, check=False,
              use_graph=use_graph)
    if inner_iters > 0:
        kw.update(inner_prec=L.TPP_FP32, flexible=True, inner_iters=inner_iters)

    def step():
        ctx.tpp_build_factors()
        x.zero_()
        return ctx.gmres_solve(b, x, **kw)[1]

    for _ in range(warmup):
        step()
    stream = torch.cuda.current_stream(device)
    torch.cuda.synchronize(device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    reps = [step() for _ in range(steps)]
    e1.record(stream)
    torch.cuda.synchronize(device)
    out = {"dim": group.dim, "n": group.n, "elements": len(group.ids), "rhs": rhs,
           "dofs": ctx.num_dofs, "ms_per_step": e0.elapsed_time(e1) / steps,
           "iters": reps[-1]["iters"], "inner_iters": reps[-1]["inner_iters"],
           "converged": all(r["converged"] for r in reps),
           "true_rel_res": reps[-1]["true_rel_res"]}
    del ctx
    return out
