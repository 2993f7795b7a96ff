"""Thin PyTorch binding of libtpp with the names of the C ABI.

Every numerical step runs in libtpp's CUDA kernels; this file only allocates
device memory with torch, converts arguments and checks status codes.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib as L


def _ptr(t: torch.Tensor) -> C.c_void_p:
    return C.c_void_p(t.data_ptr())


def _stream(stream) -> C.c_void_p:
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


class Context:
    """One DG advection problem on one GPU (a tpp_ctx and its workspace).

    velocity: a synthetic.Velocity (a_c(x) = a0_c + sum_m amp cos(2 pi k . x + phase));
    its values at the nodes and faces are evaluated on the host (mesh.py) and handed
    to the library as the arrays of tpp_problem.

    Mesh mode (batch_rhs = 0): the periodic Cartesian mesh of nel elements of width h.
    Batch mode (batch_rhs >= 1, centres [E, dim]): E isolated elements of width h
    with block-diagonal systems, batch_rhs right-hand sides each (nel is ignored);
    the field is sampled over batch_span (0: h) around each centre.  Vectors are laid
    out [element][rhs][n^dim].  ``Context.from_arrays`` takes the tpp_problem arrays
    directly.
    """

    def __init__(self, dim: int, n: int, nel, h: float, dt: float, velocity,
                 max_restart: int = 30, features: int = 0, device: str = "cuda:0",
                 stream=None, batch_rhs: int = 0, centres=None, batch_span: float = 0.0,
                 mu: int = 0):
        from . import mesh
        self.batch_rhs = int(batch_rhs)
        if self.batch_rhs > 0:
            cen = np.ascontiguousarray(centres, dtype=np.float64).reshape(-1, dim)
            self.nel = (cen.shape[0],)
            nbr, nrhs = mesh.isolated_nbr(cen.shape[0], dim), self.batch_rhs
        else:
            self.nel = tuple(int(v) for v in nel)[:dim]
            nbr, nrhs = mesh.periodic_nbr(self.nel), 1
        # geometry first (zero field): the field is evaluated at the library's
        # quadrature points (the nodes, or the mu-point rule when over-integrated)
        self._create(dim, n, nbr, nrhs, h, dt, max_restart, features, device, stream, mu)
        x = self.gauss_legendre()[0]
        if self.batch_rhs > 0:
            vn, fn = mesh.isolated_field(cen, x, velocity, batch_span if batch_span > 0 else h)
        else:
            vn, fn = mesh.periodic_field(self.nel, x, velocity)
        self.tpp_set_velocity(vn, fn, dt, stream)

    @classmethod
    def from_arrays(cls, dim: int, n: int, h: float, dt: float, nbr, vel_nodes,
                    vel_face_normal, nrhs: int = 1, max_restart: int = 30, features: int = 0,
                    device: str = "cuda:0", stream=None, mu: int = 0):
        """A context from the arrays of tpp_problem (layouts as in tpp.h)."""
        self = cls.__new__(cls)
        self.batch_rhs = 0
        nbr = np.ascontiguousarray(nbr, dtype=np.int32).reshape(-1, 2 * dim)
        self.nel = (nbr.shape[0],)
        self._create(dim, n, nbr, nrhs, h, dt, max_restart, features, device, stream, mu)
        self.tpp_set_velocity(vel_nodes, vel_face_normal, dt, stream)
        return self

    @classmethod
    def euler_system(cls, n: int, nel, h: float, dt: float, state, gamma: float = 1.4,
                     max_restart: int = 30, features: int = 0, device: str = "cuda:0",
                     stream=None):
        """The Euler equations linearised around `state` (conserved variables at the nodes,
        [E][dim + 2][n^dim], E = prod(nel) on the periodic mesh of mesh.periodic_nbr, dim =
        len(nel)): the coupled operator with the small-block preconditioners
        (tpp_create_system).  Vectors are [E][dim + 2][n^dim]; num_elem counts (element,
        component) pairs."""
        from . import mesh
        self = cls.__new__(cls)
        if not torch.cuda.is_available():
            raise RuntimeError("libtpp needs a CUDA device; there is no CPU path")
        self.lib = L.load()
        self.device = torch.device(device)
        self.batch_rhs = 0
        self.nel = tuple(int(v) for v in nel)
        dim = len(self.nel)
        self.dim, self.n, self.dt, self.h, self.nrhs, self.mu = dim, n, float(dt), float(h), 1, n
        nb = torch.as_tensor(np.ascontiguousarray(mesh.periodic_nbr(self.nel), dtype=np.int32),
                             device=self.device)
        st = torch.as_tensor(np.ascontiguousarray(state, dtype=np.float64).reshape(-1),
                             device=self.device) if not isinstance(state, torch.Tensor) \
            else state.contiguous()
        P = L.SysProblem()
        P.dim, P.n, P.num_elem, P.nc, P.flux = dim, n, int(nb.shape[0]), dim + 2, L.TPP_FLUX_EULER
        P.gamma, P.h, P.dt = float(gamma), self.h, self.dt
        P.state, P.nbr = _ptr(st), _ptr(nb)
        nbytes = self.lib.tpp_sys_workspace_bytes(C.byref(P), max_restart, features)
        if nbytes == 0:
            raise L.TppError(1, "tpp_sys_workspace_bytes")
        with torch.cuda.device(self.device):
            self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        self._ws_ptr = (self.workspace.data_ptr() + 255) & ~255
        self.ws_bytes, self.max_restart, self.features = nbytes, max_restart, features
        ctx = C.c_void_p()
        with torch.cuda.device(self.device):
            L.check(self.lib.tpp_create_system(C.byref(ctx), C.byref(P), max_restart, features,
                                               C.c_void_p(self._ws_ptr), nbytes,
                                               _stream(stream)), "tpp_create_system")
        self._ctx = ctx
        self.num_dofs = int(self.lib.tpp_num_dofs(ctx))
        self.num_elem = int(self.lib.tpp_num_elem(ctx))
        return self

    def _create(self, dim, n, nbr, nrhs, h, dt, max_restart, features, device, stream, mu=0):
        if not torch.cuda.is_available():
            raise RuntimeError("libtpp needs a CUDA device; there is no CPU path")
        self.lib = L.load()
        self.device = torch.device(device)
        self.dim, self.n, self.dt, self.h = dim, n, float(dt), float(h)
        self.nrhs = int(nrhs)
        nb = torch.as_tensor(np.ascontiguousarray(nbr, dtype=np.int32), device=self.device)
        P = L.Problem()
        P.dim, P.n, P.num_elem, P.nrhs, P.mu = dim, n, int(nb.shape[0]), self.nrhs, int(mu)
        self.mu = max(int(mu), n)
        P.h, P.dt = self.h, self.dt
        P.nbr = _ptr(nb)
        nbytes = self.lib.tpp_workspace_bytes(C.byref(P), max_restart, features)
        if nbytes == 0:
            raise L.TppError(1, "tpp_workspace_bytes")
        with torch.cuda.device(self.device):
            self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self.workspace.data_ptr()
        self._ws_ptr = (base + 255) & ~255
        self.ws_bytes = nbytes
        self.max_restart = max_restart
        self.features = features
        ctx = C.c_void_p()
        with torch.cuda.device(self.device):
            L.check(self.lib.tpp_create(C.byref(ctx), C.byref(P), max_restart, features,
                                        C.c_void_p(self._ws_ptr), nbytes, _stream(stream)),
                    "tpp_create")
        self._ctx = ctx
        self.num_dofs = int(self.lib.tpp_num_dofs(ctx))
        self.num_elem = int(self.lib.tpp_num_elem(ctx))

    def gauss_legendre(self):
        """(points, weights) of the context's quadrature rule on [0, 1] (host): the n
        Gauss-Legendre nodes, or the mu-point rule when over-integrated."""
        x, w = np.empty(self.mu), np.empty(self.mu)
        L.check(self.lib.tpp_gauss_legendre(self._ctx, x.ctypes.data_as(C.c_void_p),
                                            w.ctypes.data_as(C.c_void_p)), "tpp_gauss_legendre")
        return x, w

    def tpp_set_velocity(self, vel_nodes, vel_face_normal, dt: float, stream=None):
        """New field and step (arrays as in tpp_problem); the factors must be rebuilt."""
        vn = torch.as_tensor(np.ascontiguousarray(vel_nodes, dtype=np.float64).reshape(-1),
                             device=self.device) if not isinstance(vel_nodes, torch.Tensor) \
            else vel_nodes.contiguous()
        fn = torch.as_tensor(np.ascontiguousarray(vel_face_normal, dtype=np.float64).reshape(-1),
                             device=self.device) if not isinstance(vel_face_normal, torch.Tensor) \
            else vel_face_normal.contiguous()
        with torch.cuda.device(self.device):
            L.check(self.lib.tpp_set_velocity(self._ctx, _ptr(vn), _ptr(fn), float(dt),
                                              _stream(stream)), "tpp_set_velocity")
        self.dt = float(dt)

    def tpp_set_metric_terms(self, jdet, flux, flux_face, dt: float, stream=None):
        """Curved elements: |J_T|, |J_T| J_T^-1 a and a . |J_T| J_T^-T N^ at the quadrature
        points (layouts as in tpp.h); the factors must be rebuilt."""
        def dev(a):
            return a.contiguous() if isinstance(a, torch.Tensor) else torch.as_tensor(
                np.ascontiguousarray(a, dtype=np.float64).reshape(-1), device=self.device)
        jd, fl, ff = dev(jdet), dev(flux), dev(flux_face)
        with torch.cuda.device(self.device):
            L.check(self.lib.tpp_set_metric_terms(self._ctx, _ptr(jd), _ptr(fl), _ptr(ff),
                                                  float(dt), _stream(stream)),
                    "tpp_set_metric_terms")
        self.dt = float(dt)

    def __del__(self):
        ctx = getattr(self, "_ctx", None)
        if ctx is not None and ctx.value:
            self.lib.tpp_destroy(ctx)
            self._ctx = None

    # -- C ABI calls ---------------------------------------------------------
    def _vec(self, t, name, size=None):
        size = self.num_dofs if size is None else size
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64
                and t.is_contiguous() and t.numel() == size):
            raise ValueError(f"{name} must be a contiguous float64 CUDA tensor of {size}")
        return t

    def tpp_build_factors(self, stream=None) -> dict:
        rep = L.BuildReport()
        st = self.lib.tpp_build_factors(self._ctx, C.byref(rep), _stream(stream))
        out = {k: getattr(rep, k) for k, _ in L.BuildReport._fields_}
        out["status"] = st
        if st not in (L.TPP_OK,):
            raise L.TppError(st, "tpp_build_factors")
        return out

    def tpp_core_size(self) -> int:
        return int(self.lib.tpp_core_size(self._ctx))

    def tpp_learned_inputs(self, features: bool = True, cores: bool = True, stream=None):
        """(X [E, 2n^2+1] float32 or None, Mn [E, r*r] float64 or None, norms [E] or None)."""
        E, n, r = self.num_elem, self.n, self.tpp_core_size()
        X = torch.empty((E, 2 * n * n + 1), dtype=torch.float32, device=self.device) \
            if features else None
        Mn = torch.empty((E, r * r), dtype=torch.float64, device=self.device) if cores else None
        nr = torch.empty(E, dtype=torch.float64, device=self.device) if cores else None
        nul = C.c_void_p(0)
        L.check(self.lib.tpp_learned_inputs(self._ctx, _ptr(X) if X is not None else nul,
                                            _ptr(Mn) if Mn is not None else nul,
                                            _ptr(nr) if nr is not None else nul,
                                            _stream(stream)), "tpp_learned_inputs")
        return X, Mn, nr

    def tpp_build_factors_learned(self, net, threshold: float = 0.05, stream=None) -> dict:
        rep = L.BuildReport()
        st = self.lib.tpp_build_factors_learned(self._ctx, net._net, float(threshold),
                                                C.byref(rep), _stream(stream))
        out = {k: getattr(rep, k) for k, _ in L.BuildReport._fields_}
        out["status"] = st
        if st not in (L.TPP_OK,):
            raise L.TppError(st, "tpp_build_factors_learned")
        return out

    def tpp_solve_learned(self, net, b, x=None, threshold: float = 0.05, iter_limit: int = 50,
                          restart: int = 30, rtol: float = 1e-8, max_iters: int = 3000,
                          inner_iters: int = 0, stream=None, check: bool = True):
        """Learned build + GMRES with both fallbacks (factor error above threshold per
        element; more than iter_limit iterations: exact rebuild and continue)."""
        b = self._vec(b, "b")
        x = torch.zeros_like(b) if x is None else self._vec(x, "x")
        mixed = inner_iters > 0
        o = L.GmresOpts(restart, max_iters, rtol, L.TPP_PC_KRON,
                        L.TPP_FP32 if mixed else L.TPP_FP64, int(mixed), int(inner_iters), 0, 0.0)
        r, rep, rebuilt = L.GmresResult(), L.BuildReport(), C.c_int32(0)
        st = self.lib.tpp_solve_learned(self._ctx, net._net, float(threshold), int(iter_limit),
                                        _ptr(b), _ptr(x), C.byref(o), C.byref(r), C.byref(rep),
                                        C.byref(rebuilt), _stream(stream))
        res = {k: getattr(r, k) for k, _ in L.GmresResult._fields_}
        res["build"] = {k: getattr(rep, k) for k, _ in L.BuildReport._fields_}
        res["rebuilt"] = int(rebuilt.value)
        if check and st != L.TPP_OK:
            raise L.TppError(st, "tpp_solve_learned")
        return x, res

    def tpp_build_block_jacobi(self, stream=None):
        L.check(self.lib.tpp_build_block_jacobi(self._ctx, _stream(stream)),
                "tpp_build_block_jacobi")

    def _nrhs(self, nrhs):
        k = self.nrhs if nrhs is None else int(nrhs)
        return k, self.num_elem * k * self.n ** self.dim

    def tpp_apply_inverse(self, b, x=None, prec: int = L.TPP_FP64, stream=None, nrhs=None):
        k, size = self._nrhs(nrhs)
        b = self._vec(b, "b", size)
        x = torch.empty_like(b) if x is None else self._vec(x, "x", size)
        L.check(self.lib.tpp_apply_inverse(self._ctx, _ptr(b), _ptr(x), k, prec,
                                           _stream(stream)), "tpp_apply_inverse")
        return x

    def tpp_apply_block_jacobi(self, b, x=None, stream=None, nrhs=None):
        k, size = self._nrhs(nrhs)
        b = self._vec(b, "b", size)
        x = torch.empty_like(b) if x is None else self._vec(x, "x", size)
        L.check(self.lib.tpp_apply_block_jacobi(self._ctx, _ptr(b), _ptr(x), k, _stream(stream)),
                "tpp_apply_block_jacobi")
        return x

    def dg_apply_sumfact(self, x, y=None, stream=None, nrhs=None):
        k, size = self._nrhs(nrhs)
        x = self._vec(x, "x", size)
        y = torch.empty_like(x) if y is None else self._vec(y, "y", size)
        L.check(self.lib.dg_apply_sumfact(self._ctx, _ptr(x), _ptr(y), k, _stream(stream)),
                "dg_apply_sumfact")
        return y

    def _vec32(self, t, name, size=None):
        size = self.num_dofs if size is None else size
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32
                and t.is_contiguous() and t.numel() == size):
            raise ValueError(f"{name} must be a contiguous float32 CUDA tensor of {size}")
        return t

    def dg_apply_sumfact_f32(self, x, y=None, stream=None, nrhs=None):
        k, size = self._nrhs(nrhs)
        x = self._vec32(x, "x", size)
        y = torch.empty_like(x) if y is None else self._vec32(y, "y", size)
        L.check(self.lib.dg_apply_sumfact_f32(self._ctx, _ptr(x), _ptr(y), k, _stream(stream)),
                "dg_apply_sumfact_f32")
        return y

    def tpp_apply_inverse_f32(self, b, x=None, stream=None, nrhs=None):
        k, size = self._nrhs(nrhs)
        b = self._vec32(b, "b", size)
        x = torch.empty_like(b) if x is None else self._vec32(x, "x", size)
        L.check(self.lib.tpp_apply_inverse_f32(self._ctx, _ptr(b), _ptr(x), k, _stream(stream)),
                "tpp_apply_inverse_f32")
        return x

    def dg_apply_sumfact_static(self, x, y=None, stream=None, nrhs=None):
        """dg_apply_sumfact with its trace scratch in libtpp's static device array
        (for callers that cannot allocate device scratch; overlapping calls race)."""
        k, size = self._nrhs(nrhs)
        x = self._vec(x, "x", size)
        y = torch.empty_like(x) if y is None else self._vec(y, "y", size)
        with torch.cuda.device(self.device):
            L.check(self.lib.dg_apply_sumfact_static(self._ctx, _ptr(x), _ptr(y), k,
                                                     _stream(stream)), "dg_apply_sumfact_static")
        return y

    def gmres_solve(self, b, x=None, restart: int = 30, rtol: float = 1e-8,
                    max_iters: int = 3000, pc: int = L.TPP_PC_KRON, inner_prec: int = L.TPP_FP64,
                    flexible: bool = False, stream=None, check: bool = True,
                    inner_iters: int = 0, inner_rtol: float = 0.0, use_graph: bool = False):
        b = self._vec(b, "b")
        x = torch.zeros_like(b) if x is None else self._vec(x, "x")
        o = L.GmresOpts(restart, max_iters, rtol, pc, inner_prec, int(flexible), int(inner_iters),
                        int(use_graph), float(inner_rtol))
        r = L.GmresResult()
        st = self.lib.gmres_solve(self._ctx, _ptr(b), _ptr(x), C.byref(o), C.byref(r),
                                  _stream(stream))
        res = {k: getattr(r, k) for k, _ in L.GmresResult._fields_}
        if check and st != L.TPP_OK:
            raise L.TppError(st, "gmres_solve")
        return x, res

    def tpp_time_integrate(self, u, scheme: int, dt: float, steps: int,
                           rebuild_each_step: bool = False, restart: int = 30, rtol: float = 1e-10,
                           max_iters: int = 3000, pc: int = L.TPP_PC_KRON, use_graph: bool = False,
                           inner_iters: int = 0, stream=None, check: bool = True) -> dict:
        """Advance u (float64 CUDA tensor, in place) by `steps` steps of `scheme`
        (TPP_TS_*); implicit stages by GMRES with these options.  Implicit schemes leave
        the context's operator at dt_ctx = a_ii dt.  Returns the report."""
        u = self._vec(u, "u")
        mixed = inner_iters > 0
        o = L.GmresOpts(restart, max_iters, rtol, pc, L.TPP_FP32 if mixed else L.TPP_FP64,
                        int(mixed), int(inner_iters), int(use_graph), 0.0)
        rep = L.TimeReport()
        with torch.cuda.device(self.device):
            st = self.lib.tpp_time_integrate(self._ctx, _ptr(u), int(scheme), float(dt), int(steps),
                                             int(bool(rebuild_each_step)), C.byref(o),
                                             C.byref(rep), _stream(stream))
        out = {k: getattr(rep, k) for k, _ in L.TimeReport._fields_}
        out["status"] = st
        if check and st != L.TPP_OK:
            raise L.TppError(st, "tpp_time_integrate")
        return out

    def tpp_mass_solve(self, mu: int, jac_q, jac_n, r, x=None, rtol: float = 1e-12,
                       max_iters: int = 100, nrhs=None, stream=None, check: bool = True):
        """Element-wise PCG solve of M_K x = r with the mu-point exact mass matrix
        (jac_q [E, mu^dim], jac_n [E, n^dim]: |J_T| at the quadrature points and nodes).
        Returns (x, iterations per block [E * nrhs] int32 tensor, status)."""
        k, size = self._nrhs(nrhs)
        r = self._vec(r, "r", size)
        x = torch.empty_like(r) if x is None else self._vec(x, "x", size)
        jq = torch.as_tensor(np.ascontiguousarray(jac_q, dtype=np.float64).reshape(-1),
                             device=self.device)
        jn = torch.as_tensor(np.ascontiguousarray(jac_n, dtype=np.float64).reshape(-1),
                             device=self.device)
        if jq.numel() != self.num_elem * mu ** self.dim or jn.numel() != self.num_elem * self.n ** self.dim:
            raise ValueError("jac_q must hold E mu^dim values and jac_n E n^dim")
        its = torch.zeros(self.num_elem * k, dtype=torch.int32, device=self.device)
        with torch.cuda.device(self.device):
            st = self.lib.tpp_mass_solve(self._ctx, int(mu), _ptr(jq), _ptr(jn), _ptr(r), _ptr(x),
                                         k, float(rtol), int(max_iters), _ptr(its),
                                         _stream(stream))
        if check and st != L.TPP_OK:
            raise L.TppError(st, "tpp_mass_solve")
        return x, its, st

    def views(self) -> dict:
        """Copies of the factor arrays (torch tensors) for inspection."""
        v = L.Views()
        L.check(self.lib.tpp_get_views(self._ctx, C.byref(v)), "tpp_get_views")
        E, n = self.num_elem, self.n
        torch.cuda.synchronize(self.device)

        def grab(addr, count, dtype):
            if not addr:
                return None                    # array absent in this form / dimension
            out = torch.empty(count, dtype=dtype, device=self.device)
            L.check(self.lib.tpp_copy_device(_ptr(out), C.c_void_p(addr),
                                             count * out.element_size(), _stream(None)),
                    "tpp_copy_device")
            return out

        res = {"sigma": grab(v.sigma, 2 * E, torch.float64).view(E, 2)}
        for name in ("A1", "B1", "A2", "B2", "SA", "SB", "Q1", "Q2", "T1", "T2"):
            # column-major n x n per element -> [E, n, n] with [e, row, col]
            t = grab(getattr(v, name), E * n * n, torch.float64)
            res[name] = None if t is None else t.view(E, n, n).transpose(1, 2)
        res["G"] = grab(v.G, E * 2 * n ** 3, torch.float64)   # one-sided shifted inverses
        res["flags"] = grab(v.flags, E, torch.int32)
        res["cond"] = grab(v.cond, E, torch.float64)
        res["gl_x"] = grab(v.gl_x, n, torch.float64)
        res["gl_w"] = grab(v.gl_w, n, torch.float64)
        res["D"] = grab(v.D, n * n, torch.float64).view(n, n)
        if self.mu > self.n:
            r, m = self.tpp_core_size(), 2 * self.mu + 2
            res["core"] = grab(v.core, E * r * r, torch.float64).view(E, r, r).transpose(1, 2)
            res["Qb"] = grab(v.Qb, n * n * r, torch.float64).view(r, n * n).t()
            res["Rb"] = grab(v.Rb, r * m, torch.float64).view(r, m)
            res["qtr"] = grab(v.qtr, r, torch.float64)
        if self.dim == 3:
            res["Az"] = grab(v.Az, E * n * n, torch.float64).view(E, n, n).transpose(1, 2)
            res["Azi"] = grab(v.Azi, E * n * n, torch.float64).view(E, n, n).transpose(1, 2)
            res["sigz"] = grab(v.sigz, E, torch.float64)
            res["zflags"] = grab(v.zflags, E, torch.int32)
        if v.fA:                       # full multi-component blocks (row-major factors)
            Ep, m = self.num_elem // (self.dim + 2), (self.dim + 2) * n
            if self.dim == 2:          # A_k, B_k of A_1 (x) B_1 + A_2 (x) B_2
                res["fA"] = grab(v.fA, Ep * 2 * m * m, torch.float64).view(Ep, 2, m, m)
                res["fB"] = grab(v.fB, Ep * 2 * n * n, torch.float64).view(Ep, 2, n, n)
            else:                      # first-stage A_1; the y-x factors are A1/B1/A2/B2[:Ep]
                res["fA"] = grab(v.fA, Ep * m * m, torch.float64).view(Ep, m, m)
            res["fsig"] = grab(v.fsig, Ep * 2, torch.float64).view(Ep, 2)
            res["fflags"] = grab(v.fflags, Ep, torch.int32)
        torch.cuda.synchronize(self.device)
        return res


