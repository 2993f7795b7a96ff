"""Mixed-degree batches of block-diagonal DG advection systems.

Each element of the batch is isolated (its system is its own diagonal block:
mass, volume and outflow face terms, no neighbour coupling) and carries R
right-hand sides.  Elements are grouped by (dimension, n); each group is one
libtpp context in batch mode, so every kernel of a group runs with one degree
and the factor build, the Kronecker apply and the Krylov solve treat all the
group's systems at once.  Groups run one after another on the caller's stream.
BatchGmres solves every (element, right-hand side) system with its own GMRES
in persistent launches over all groups (tpp_batch_gmres).  This module only
sequences calls to the C ABI (through Context).
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


class BatchGmres:
    """Per-system GMRES over isolated-element contexts in persistent launches
    grouped by n (tpp_batch_gmres): every (element, right-hand side) system has
    its own Arnoldi process and convergence test.  The contexts must be isolated,
    two-sided (TPP_FEAT_TWO_SIDED) and have their factors built before solve();
    mixed=True also needs TPP_FEAT_MIXED.  The workspace is sized once here and
    reused by every solve()."""

    def __init__(self, contexts, *, restart: int = 20, rtol: float = 1e-8,
                 max_iters: int = 300, mixed: bool = False, inner_rtol: float = 1e-4,
                 max_outer: int = 8, warps=(0, 0, 0), ctas_per_sm=(0, 0, 0),
                 reg_budget=(0, 0, 0), per_system: bool = False):
        import ctypes as C
        self.C = C
        self.lib = L.load()
        self.contexts = list(contexts)
        self.device = self.contexts[0].device
        k = len(self.contexts)
        self._ctxs = (C.c_void_p * k)(*[c._ctx.value for c in self.contexts])
        self.iters = self.relres = None
        o = L.BatchOpts()
        o.restart, o.max_iters, o.rtol = int(restart), int(max_iters), float(rtol)
        o.prec = L.TPP_FP32 if mixed else L.TPP_FP64
        o.max_outer, o.inner_rtol = int(max_outer), float(inner_rtol)
        for i in range(3):
            o.warps[i], o.ctas_per_sm[i] = int(warps[i]), int(ctas_per_sm[i])
            o.reg_budget[i] = int(reg_budget[i])
        if per_system:
            sizes = [c.num_dofs // c.n ** c.dim for c in self.contexts]
            self.iters = [torch.zeros(m, dtype=torch.int32, device=self.device) for m in sizes]
            self.relres = [torch.zeros(m, dtype=torch.float64, device=self.device) for m in sizes]
            self._ip = (C.c_void_p * k)(*[t.data_ptr() for t in self.iters])
            self._rp = (C.c_void_p * k)(*[t.data_ptr() for t in self.relres])
            o.iters = C.cast(self._ip, C.c_void_p)
            o.relres = C.cast(self._rp, C.c_void_p)
        self.opts = o
        with torch.cuda.device(self.device):
            nbytes = self.lib.tpp_batch_workspace_bytes(self._ctxs, k, C.byref(o))
        if nbytes == 0:
            raise L.TppError(1, "tpp_batch_workspace_bytes")
        self.ws = torch.empty(int(nbytes), dtype=torch.uint8, device=self.device)

    def solve(self, bs, xs, stream=None, check: bool = True) -> dict:
        """x_g = S^-1 b_g system by system (zero initial guess); bs, xs: float64 CUDA
        tensors [E][nrhs][n^d], one pair per context.  Returns the report as a dict."""
        C = self.C
        k = len(self.contexts)
        for c, b, x in zip(self.contexts, bs, xs):
            c._vec(b, "b")
            c._vec(x, "x")
        bp = (C.c_void_p * k)(*[b.data_ptr() for b in bs])
        xp = (C.c_void_p * k)(*[x.data_ptr() for x in xs])
        rep = L.BatchReport()
        s = torch.cuda.current_stream(self.device) if stream is None else stream
        with torch.cuda.device(self.device):
            st = self.lib.tpp_batch_gmres(self._ctxs, k, bp, xp, C.byref(self.opts),
                                          C.byref(rep), C.c_void_p(self.ws.data_ptr()),
                                          self.ws.numel(), C.c_void_p(s.cuda_stream))
        out = {f: getattr(rep, f) for f, _ in L.BatchReport._fields_}
        out["launch_ms"] = list(rep.launch_ms)
        out["status"] = st
        if check and st != L.TPP_OK:
            raise L.TppError(st, "tpp_batch_gmres")
        return out
