"""DG discretisation of linear advection, assembled explicitly (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The conservation law u_t + div(a u) = 0 (Sec. 5.1, Eq. adv) is discretised
with the weak form of Eq. weak-form on a periodic Cartesian mesh of N^d
elements of width h.  An implicit step gives (M - dt J) x = b (Sec. 3.4); we
write S = M - dt J = M + dt A with A = -J.

Element blocks are assembled from the Kronecker forms of Table tab:dg-ops
and Eq. mass-kron / adv-kron: mass (G^T W)^{(x)d} J_T G^{(x)d}, volume
-dt (G^T W (x) D^T W) F_1 (G (x) G) - dt (D^T W (x) G^T W) F_2 (G (x) G) in 2D
(and the three-term analogue in 3D).  For the affine Cartesian map x = x0 + h xi
the Jacobian determinant is J_T = h^d and the reference-space flux Jacobians are
F_c = h^(d-1) diag(a_c at the quadrature points).  Face terms follow the face
sum of Eq. jac-entries with the upwind flux F^ = (a.n) u^- if a.n >= 0 else
(a.n) u^+ (reading of the generic numerical flux of Sec. 2), so the diagonal
block gets dt h^(d-1) E_f^T diag(w_f max(a.n, 0)) E_f and the neighbour block
dt h^(d-1) E_f^T diag(w_f min(a.n, 0)) E'_f, with E_f (E'_f) the own
(neighbour) basis evaluated at the face quadrature points.

The velocity is a field on the periodic domain [0, L_1] x ... with
L_d = N_d h: it is evaluated at the normalised point x / L (a function of
the unit cube), so it is periodic on the mesh whatever h is.

DOF ordering: element-major, inside an element i + n j (+ n^2 k), x fastest,
so the slowest direction is the LEFT Kronecker factor.  Face order: -x, +x,
-y, +y, -z, +z.  The physical coordinate of a face is taken from the element
that owns it as its lower face (wrapped periodically), so both sides of every
face evaluate the velocity at bit-identical points.

Pinned in tests/test_oracle_dg.py: the n = 1 finite-volume closed form,
A 1 = 0 for constant velocity, discrete conservation 1^T A x = 0 for any
velocity, exact mass and constant-velocity volume integrals against a
higher-order quadrature, and agreement of the explicit assembly with the
sum-factorised matvec (Alg. matrix-free-matvec) written independently below.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp

from .basis import Basis1D


def velocity_eval(vel, X: np.ndarray) -> np.ndarray:
    """a_c(X) for points X[..., dim]; returns [..., dim]."""
    X = np.asarray(X, dtype=np.float64)
    out = np.empty(X.shape[:-1] + (vel.dim,))
    for c in range(vel.dim):
        val = np.full(X.shape[:-1], float(vel.a0[c]))
        for m in range(vel.n_modes):
            arg = 2.0 * np.pi * (X @ vel.kvec[c, m].astype(np.float64)) + vel.phase[c, m]
            val = val + vel.amp[c, m] * np.cos(arg)
        out[..., c] = val
    return out


class PeriodicMesh:
    """N_1 x ... x N_d periodic Cartesian mesh of the unit cube (or of width h)."""

    def __init__(self, nel, h: float | None = None):
        self.nel = tuple(int(v) for v in nel)
        self.dim = len(self.nel)
        self.h = 1.0 / self.nel[0] if h is None else float(h)
        self.num_elem = int(np.prod(self.nel))

    def coords(self, e: int):
        c = []
        for N in self.nel:
            c.append(e % N)
            e //= N
        return tuple(c)

    def index(self, c) -> int:
        e, stride = 0, 1
        for ci, N in zip(c, self.nel):
            e += (ci % N) * stride
            stride *= N
        return e

    def neighbor(self, e: int, face: int) -> int:
        c = list(self.coords(e))
        d, side = divmod(face, 2)
        c[d] += 1 if side == 1 else -1
        return self.index(c)


def _kron_all(mats):
    out = mats[0]
    for m in mats[1:]:
        out = np.kron(out, m)
    return out


class AdvectionDG:
    """S = M + dt A for linear advection on a periodic mesh (oracle form)."""

    def __init__(self, mesh: PeriodicMesh, n: int, dt: float, vel, mu: int | None = None):
        assert vel.dim == mesh.dim
        self.mesh, self.dim, self.n, self.dt, self.vel = mesh, mesh.dim, n, float(dt), vel
        self.basis = Basis1D(n, mu)
        self.nloc = n ** self.dim
        self.ndof = mesh.num_elem * self.nloc

    # -- quadrature points ---------------------------------------------------
    def volume_points(self, e: int) -> np.ndarray:
        """Physical quadrature points, index a + mu b (+ mu^2 c), x fastest."""
        c = self.mesh.coords(e)
        x = self.basis.x
        grids = np.meshgrid(*([x] * self.dim), indexing="ij")   # grids[d][a,b,(c)]
        pts = np.stack([(c[d] + grids[d]) * self.mesh.h for d in range(self.dim)], axis=-1)
        # flatten with x fastest: transpose axes so the x index is last
        pts = np.transpose(pts, tuple(range(self.dim - 1, -1, -1)) + (self.dim,))
        return pts.reshape(-1, self.dim)

    def face_points(self, e: int, face: int) -> np.ndarray:
        """Physical points on face `face` of element e (tangential x fastest)."""
        d, side = divmod(face, 2)
        c = list(self.mesh.coords(e))
        x = self.basis.x
        tang = [t for t in range(self.dim) if t != d]
        grids = np.meshgrid(*([x] * (self.dim - 1)), indexing="ij") if self.dim > 1 else []
        owner = (c[d] + side) % self.mesh.nel[d]       # element owning this face as its lower face
        cols = []
        for t in range(self.dim):
            if t == d:
                cols.append(None)
            else:
                k = tang.index(t)
                cols.append((c[t] + grids[k]) * self.mesh.h)
        shape = grids[0].shape
        pts = np.empty(shape + (self.dim,))
        for t in range(self.dim):
            pts[..., t] = owner * self.mesh.h if t == d else cols[t]
        pts = np.transpose(pts, tuple(range(self.dim - 2, -1, -1)) + (self.dim - 1,))
        return pts.reshape(-1, self.dim)

    # -- Kronecker building blocks (Table tab:dg-ops) ------------------------
    def _face_eval(self, face: int, own: bool = True) -> np.ndarray:
        """E[q, I]: element basis at the face quadrature points of `face`.

        own=False evaluates the neighbour's basis at the same physical points
        (the neighbour sees the face on its opposite side)."""
        b = self.basis
        d, side = divmod(face, 2)
        if not own:
            side = 1 - side
        lvec = (b.l1 if side == 1 else b.l0)[None, :]
        mats = []
        for t in range(self.dim - 1, -1, -1):      # slowest direction first
            mats.append(lvec if t == d else b.G)
        return _kron_all(mats)

    def _face_weights(self) -> np.ndarray:
        w = self.basis.w
        return _kron_all([w] * (self.dim - 1)) if self.dim > 1 else np.ones(1)

    def domain_length(self) -> np.ndarray:
        return np.array([N * self.mesh.h for N in self.mesh.nel])

    def velocity_at(self, X: np.ndarray) -> np.ndarray:
        """a at physical points X (field defined on the normalised domain)."""
        return velocity_eval(self.vel, X / self.domain_length())

    def face_normal_velocity(self, e: int, face: int) -> np.ndarray:
        d, side = divmod(face, 2)
        a = self.velocity_at(self.face_points(e, face))
        return a[:, d] * (1.0 if side == 1 else -1.0)

    def mass_block(self, e: int) -> np.ndarray:
        b = self.basis
        GtW = b.G.T @ b.W
        JT = np.diag(np.full(b.mu ** self.dim, self.mesh.h ** self.dim))
        G = _kron_all([b.G] * self.dim)
        return _kron_all([GtW] * self.dim) @ JT @ G

    def volume_jacobian_block(self, e: int) -> np.ndarray:
        """J_v: derivative of int F(u) . grad v dx (Table tab:dg-ops, Eq. adv-kron)."""
        b = self.basis
        GtW, DtW = b.G.T @ b.W, b.D.T @ b.W
        a = self.velocity_at(self.volume_points(e))
        G = _kron_all([b.G] * self.dim)
        Jv = np.zeros((self.nloc, self.nloc))
        for comp in range(self.dim):
            Fc = np.diag(self.mesh.h ** (self.dim - 1) * a[:, comp])
            mats = [DtW if t == comp else GtW for t in range(self.dim - 1, -1, -1)]
            Jv += _kron_all(mats) @ Fc @ G
        return Jv

    def face_blocks(self, e: int):
        """Diagonal-block face term and the neighbour coupling blocks.

        Returns (Fdiag, {face: (nbr, Fnbr)}) such that the face part of
        A = -J contributes Fdiag x_e + sum_f Fnbr_f x_nbr(f) to row block e."""
        hf = self.mesh.h ** (self.dim - 1)
        wf = self._face_weights()
        Fdiag = np.zeros((self.nloc, self.nloc))
        nbrs = {}
        for face in range(2 * self.dim):
            an = self.face_normal_velocity(e, face)
            E = self._face_eval(face, own=True)
            En = self._face_eval(face, own=False)
            Fdiag += hf * E.T @ np.diag(wf * np.maximum(an, 0.0)) @ E
            nbrs[face] = (self.mesh.neighbor(e, face),
                          hf * E.T @ np.diag(wf * np.minimum(an, 0.0)) @ En)
        return Fdiag, nbrs

    def element_block(self, e: int) -> np.ndarray:
        """Diagonal block S_e = M_e - dt (J_v + J_f)_e."""
        Fdiag, _ = self.face_blocks(e)
        return self.mass_block(e) - self.dt * self.volume_jacobian_block(e) + self.dt * Fdiag

    def global_matrix(self) -> sp.csr_matrix:
        nl = self.nloc
        rows, cols, vals = [], [], []
        for e in range(self.mesh.num_elem):
            Fdiag, nbrs = self.face_blocks(e)
            blocks = [(e, self.mass_block(e) - self.dt * self.volume_jacobian_block(e)
                       + self.dt * Fdiag)]
            for face, (nb, Fn) in nbrs.items():
                blocks.append((nb, self.dt * Fn))
            for col_e, B in blocks:
                r, c = np.nonzero(B)
                rows.append(e * nl + r)
                cols.append(col_e * nl + c)
                vals.append(B[r, c])
        rows, cols, vals = (np.concatenate(v) for v in (rows, cols, vals))
        return sp.csr_matrix((vals, (rows, cols)), shape=(self.ndof, self.ndof))

    # -- sum-factorised matvec (Alg. matrix-free-matvec, Eq. after jac-entries)
    def apply_sumfact(self, x: np.ndarray) -> np.ndarray:
        """y = (M - dt J) x element by element with one-dimensional contractions.

        Written independently of the explicit assembly: the solution is
        evaluated at quadrature points by d successive 1D contractions with G,
        multiplied by the point-wise weights / flux Jacobians, and integrated
        back with G^T W or D^T W along each direction."""
        b, d, n, mu, h = self.basis, self.dim, self.n, self.basis.mu, self.mesh.h
        X = x.reshape(self.mesh.num_elem, *([n] * d))  # axes: (e, [z], y, x)
        y = np.zeros_like(X)
        wq = _kron_all([b.w] * d).reshape([mu] * d)

        def contract(T, Mat, axis):
            # T[..., j along axis, ...] -> sum_j Mat[a, j] T[..., j, ...]
            T = np.moveaxis(T, axis, -1)
            T = T @ Mat.T
            return np.moveaxis(T, -1, axis)

        for e in range(self.mesh.num_elem):
            u = X[e]
            for ax in range(d):
                u = contract(u, b.G, ax)                # values at quadrature points
            a = self.velocity_at(self.volume_points(e)).reshape([mu] * d + [d])
            ye = np.zeros([n] * d)
            # mass
            t = u * wq * h ** d
            for ax in range(d):
                t = contract(t, b.G.T, ax)
            ye += t
            # volume: component c differentiates along its own axis
            for comp in range(d):
                ax_c = d - 1 - comp                      # x is the last axis
                t = u * wq * a[..., comp] * h ** (d - 1)
                for ax in range(d):
                    t = contract(t, b.D.T if ax == ax_c else b.G.T, ax)
                ye -= self.dt * t
            # faces
            wf = self._face_weights()
            for face in range(2 * d):
                nb = self.mesh.neighbor(e, face)
                an = self.face_normal_velocity(e, face)
                E, En = self._face_eval(face, True), self._face_eval(face, False)
                flux = np.maximum(an, 0) * (E @ X[e].reshape(-1)) + \
                    np.minimum(an, 0) * (En @ X[nb].reshape(-1))
                ye += self.dt * h ** (d - 1) * (E.T @ (wf * flux)).reshape([n] * d)
            y[e] = ye
        return y.reshape(-1)


class IsolatedElements:
    """Block-diagonal systems of a batch of isolated elements (oracle form).

    Element e is the cube [c_e - h/2, c_e + h/2]^d of the unit domain (centre
    c_e); its system is the diagonal block S_e = M_e + dt (A_v + A_f)_e of the
    DG discretisation above with every neighbour coupling dropped: mass,
    volume, and the own-side upwind face terms dt h^(d-1) E_f^T diag(w_f
    max(a.n, 0)) E_f on all 2d faces (Eq. jac-entries).  The velocity is the
    field at the point c_e + span (xi - 1/2) of the unit domain (span = h unless
    given): the element's integrals scale with its width h, the field is sampled
    over span.  Per element these are the diagonal blocks of the periodic-mesh
    operator (span = 1/N), which pins this class against
    AdvectionDG.element_block in tests/test_oracle_dg.py.
    """

    def __init__(self, n: int, h: float, centres: np.ndarray, dt: float, vel,
                 span: float | None = None):
        self.centres = np.asarray(centres, dtype=np.float64)
        self.dim = self.centres.shape[1]
        assert vel.dim == self.dim
        self.n, self.h, self.dt, self.vel = n, float(h), float(dt), vel
        self.span = float(h if span is None else span)
        self.basis = Basis1D(n)
        self.nloc = n ** self.dim
        self.num_elem = self.centres.shape[0]

    def _grid(self, lo: np.ndarray) -> np.ndarray:
        """Points lo + span x at the tensor nodes, index a + n b (+ n^2 c), x fastest."""
        x = self.basis.x
        grids = np.meshgrid(*([x] * self.dim), indexing="ij")
        pts = np.stack([lo[d] + self.span * grids[d] for d in range(self.dim)], axis=-1)
        pts = np.transpose(pts, tuple(range(self.dim - 1, -1, -1)) + (self.dim,))
        return pts.reshape(-1, self.dim)

    def block(self, e: int) -> np.ndarray:
        b, d, h, sp = self.basis, self.dim, self.h, self.span
        lo = self.centres[e] - 0.5 * sp
        a = velocity_eval(self.vel, self._grid(lo))
        GtW, DtW = b.G.T @ b.W, b.D.T @ b.W
        G = _kron_all([b.G] * d)
        S = _kron_all([GtW] * d) @ np.diag(np.full(self.nloc, h ** d)) @ G
        for comp in range(d):
            mats = [DtW if t == comp else GtW for t in range(d - 1, -1, -1)]
            S -= self.dt * _kron_all(mats) @ np.diag(h ** (d - 1) * a[:, comp]) @ G
        # faces: tangential nodes x fastest, the normal coordinate at the face
        x = b.x
        wf = _kron_all([b.w] * (d - 1)) if d > 1 else np.ones(1)
        for face in range(2 * d):
            dn, side = divmod(face, 2)
            tang = [t for t in range(d) if t != dn]
            grids = np.meshgrid(*([x] * (d - 1)), indexing="ij") if d > 1 else []
            pts = np.empty((grids[0].shape if d > 1 else ()) + (d,))
            for t in range(d):
                pts[..., t] = (lo[t] + side * sp) if t == dn else lo[t] + sp * grids[tang.index(t)]
            pts = np.transpose(pts, tuple(range(d - 2, -1, -1)) + (d - 1,)).reshape(-1, d)
            an = velocity_eval(self.vel, pts)[:, dn] * (1.0 if side == 1 else -1.0)
            lvec = (b.l1 if side == 1 else b.l0)[None, :]
            E = _kron_all([lvec if t == dn else b.G for t in range(d - 1, -1, -1)])
            S += self.dt * h ** (d - 1) * E.T @ np.diag(wf * np.maximum(an, 0.0)) @ E
        return S
