"""Linearised DG operator of a system of conservation laws in 2D and 3D (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Sec. 5.3 and Sec. 5.6: for the Euler equations the unknowns have n_c components
(n_c = 4 in 2D: rho, rho u, rho v, rho E, flux of Eq. euler-flux; n_c = 5 in 3D with
the third momentum), so the diagonal blocks of the Jacobian are n_c n^d x n_c n^d
("full" blocks); the "small" blocks are their n_c diagonal n^d x n^d sub-blocks,
which do not couple the components.

The DG discretisation is the one of oracle/dg.py (collocated Gauss-Legendre nodes,
periodic Cartesian mesh of square elements of width h) applied to every
component, with the local Lax-Friedrichs numerical flux
  F^(u-, u+) . n = 1/2 (F(u-) + F(u+)) . n + 1/2 lam (u- - u+),
  lam = max(|v- . n| + c-, |v+ . n| + c+)
(the generic numerical flux of Sec. 2; the paper does not name the one used for
Euler).  Linearised around a DG state u0 (its nodal values; traces by the face
evaluation matrices) with lam frozen at its value for u0, the residual's
Jacobian has
  volume   -dt sum_d K_d diag(h^(d-1) A_d[c, c'](u0)) G   (K_d: D^T W in direction d,
                                                         G^T W in the others)
  faces    own:  dt h^(d-1) E^T diag(w_f 1/2 (A_n(u0-)[c, c'] + lam delta_cc')) E
           nbr:  dt h^(d-1) E^T diag(w_f 1/2 (A_n(u0+)[c, c'] - lam delta_cc')) E'
with A_d = dF_d/du and A_n = sum_d n_d A_d for the outward normal n.
S = M - dt J as in oracle/dg.py.  DOF ordering: element, then component, then
node i + n j (+ n^2 k) (x fastest).

Pinned in tests/test_oracle_systems.py: the analytic Euler Jacobians against
finite differences of the flux, the eigenvalues of A_n (v.n - c, v.n, v.n,
v.n + c), the reduction of a one-component linear "system" (flux a u, lam =
|a.n|) to the upwind advection operator of oracle/dg.py, discrete conservation of
every component, and J x against a finite difference of the nonlinear DG residual;
the full-block KSVD (2D) and nested KSVD (3D) against the scalar ones for one component
and against an exact Kronecker block (dt = 0: the mass alone).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .dg import AdvectionDG, PeriodicMesh, _kron_all


# ---- 2D Euler (Eq. euler-flux) --------------------------------------------------
def euler_primitive(U: np.ndarray, gamma: float):
    rho = U[..., 0]
    u, v = U[..., 1] / rho, U[..., 2] / rho
    p = (gamma - 1.0) * (U[..., 3] - 0.5 * rho * (u * u + v * v))
    H = (U[..., 3] + p) / rho
    return rho, u, v, p, H


def euler_flux(U: np.ndarray, gamma: float):
    """(F_1, F_2) of Eq. euler-flux, each [..., 4]."""
    rho, u, v, p, H = euler_primitive(U, gamma)
    F1 = np.stack([rho * u, rho * u * u + p, rho * u * v, rho * H * u], axis=-1)
    F2 = np.stack([rho * v, rho * u * v, rho * v * v + p, rho * H * v], axis=-1)
    return F1, F2


def euler_jacobians(U: np.ndarray, gamma: float):
    """A_x = dF_1/dU, A_y = dF_2/dU in conserved variables, each [..., 4, 4]
    (derived by differentiating Eq. euler-flux; pinned by finite differences)."""
    rho, u, v, p, H = euler_primitive(U, gamma)
    g1 = gamma - 1.0
    phi = 0.5 * g1 * (u * u + v * v)
    z, o = np.zeros_like(u), np.ones_like(u)
    Ax = np.stack([
        np.stack([z, o, z, z], -1),
        np.stack([phi - u * u, (3.0 - gamma) * u, -g1 * v, g1 * o], -1),
        np.stack([-u * v, v, u, z], -1),
        np.stack([u * (phi - H), H - g1 * u * u, -g1 * u * v, gamma * u], -1)], -2)
    Ay = np.stack([
        np.stack([z, z, o, z], -1),
        np.stack([-u * v, v, u, z], -1),
        np.stack([phi - v * v, -g1 * u, (3.0 - gamma) * v, g1 * o], -1),
        np.stack([v * (phi - H), -g1 * u * v, H - g1 * v * v, gamma * v], -1)], -2)
    return Ax, Ay


def euler_wave_speed(U: np.ndarray, nvec, gamma: float) -> np.ndarray:
    """|v.n| + c (the largest |eigenvalue| of A_n)."""
    rho, u, v, p, H = euler_primitive(U, gamma)
    return np.abs(u * nvec[0] + v * nvec[1]) + np.sqrt(gamma * p / rho)


# ---- 3D Euler (Eq. euler-flux with a third momentum component) -----------------
def euler3d_flux(U: np.ndarray, gamma: float):
    """(F_1, F_2, F_3), each [..., 5], for U = (rho, rho u, rho v, rho w, rho E)."""
    rho = U[..., 0]
    V = U[..., 1:4] / rho[..., None]
    p = (gamma - 1.0) * (U[..., 4] - 0.5 * rho * np.sum(V * V, -1))
    H = (U[..., 4] + p) / rho
    out = []
    for d in range(3):
        vd = V[..., d]
        mom = [rho * V[..., i] * vd + (p if i == d else 0.0) for i in range(3)]
        out.append(np.stack([rho * vd] + mom + [rho * H * vd], -1))
    return tuple(out)


def euler3d_jacobians(U: np.ndarray, gamma: float):
    """A_d = dF_d/dU, d = x, y, z, each [..., 5, 5] (derived from euler3d_flux; pinned by
    finite differences)."""
    rho = U[..., 0]
    V = U[..., 1:4] / rho[..., None]
    q2 = np.sum(V * V, -1)
    g1 = gamma - 1.0
    p = g1 * (U[..., 4] - 0.5 * rho * q2)
    H = (U[..., 4] + p) / rho
    phi = 0.5 * g1 * q2
    mats = []
    for d in range(3):
        A = np.zeros(U.shape[:-1] + (5, 5))
        vd = V[..., d]
        A[..., 0, 1 + d] = 1.0
        for i in range(3):
            A[..., 1 + i, 0] = -V[..., i] * vd + (phi if i == d else 0.0)
            for j in range(3):
                A[..., 1 + i, 1 + j] = ((vd if i == j else 0.0) + (V[..., i] if j == d else 0.0)
                                        - (g1 * V[..., j] if i == d else 0.0))
            A[..., 1 + i, 4] = g1 if i == d else 0.0
        A[..., 4, 0] = vd * (phi - H)
        for j in range(3):
            A[..., 4, 1 + j] = (H if j == d else 0.0) - g1 * V[..., j] * vd
        A[..., 4, 4] = gamma * vd
        mats.append(A)
    return tuple(mats)


def euler3d_wave_speed(U: np.ndarray, nvec, gamma: float) -> np.ndarray:
    rho = U[..., 0]
    V = U[..., 1:4] / rho[..., None]
    p = (gamma - 1.0) * (U[..., 4] - 0.5 * rho * np.sum(V * V, -1))
    return np.abs(V @ np.asarray(nvec, dtype=np.float64)) + np.sqrt(gamma * p / rho)


class Euler3DFlux:
    nc, dim = 5, 3

    def __init__(self, gamma: float = 1.4):
        self.gamma = gamma

    def flux(self, U):
        return euler3d_flux(U, self.gamma)

    def jacobians(self, U):
        return euler3d_jacobians(U, self.gamma)

    def speed(self, U, nvec):
        return euler3d_wave_speed(U, nvec, self.gamma)


class EulerFlux:
    nc, dim = 4, 2

    def __init__(self, gamma: float = 1.4):
        self.gamma = gamma

    def flux(self, U):
        return euler_flux(U, self.gamma)

    def jacobians(self, U):
        return euler_jacobians(U, self.gamma)

    def speed(self, U, nvec):
        return euler_wave_speed(U, nvec, self.gamma)


class LinearAdvectionFlux:
    """One-component linear 'system' F(u) = a u with a constant velocity a (for the
    reduction pin against oracle/dg.py), in 2D or 3D."""
    nc = 1

    def __init__(self, a):
        self.a = np.asarray(a, dtype=np.float64)
        self.dim = len(self.a)

    def flux(self, U):
        return tuple(self.a[d] * U for d in range(self.dim))

    def jacobians(self, U):
        shp = U.shape[:-1] + (1, 1)
        return tuple(np.full(shp, self.a[d]) for d in range(self.dim))

    def speed(self, U, nvec):
        return np.full(U.shape[:-1], abs(float(np.dot(self.a, nvec))))


def normals(dim: int):
    """Outward normals of the faces -x, +x, -y, +y (, -z, +z)."""
    out = []
    for d in range(dim):
        for side in (-1.0, 1.0):
            v = [0.0] * dim
            v[d] = side
            out.append(tuple(v))
    return tuple(out)


NORMALS = normals(2)


class LinearizedSystemDG:
    """S = M - dt J of a system linearised around the nodal state U0 [E, nc, n^d]."""

    def __init__(self, mesh: PeriodicMesh, n: int, dt: float, flux, U0: np.ndarray):
        self.mesh, self.n, self.dt, self.flux = mesh, n, float(dt), flux
        self.dim = mesh.dim
        assert getattr(flux, "dim", self.dim) == self.dim
        self.nc = flux.nc
        self.scalar = AdvectionDG(mesh, n, dt, _ZeroVelocity(self.dim))   # basis, face matrices
        self.basis = self.scalar.basis
        self.nloc = n ** self.dim
        self.bs = self.nc * self.nloc                 # block size
        self.ndof = mesh.num_elem * self.bs
        self.hf = mesh.h ** (self.dim - 1)
        self.normals = normals(self.dim)
        self.U0 = np.asarray(U0, dtype=np.float64).reshape(mesh.num_elem, self.nc, self.nloc)

    # -- linearisation data -------------------------------------------------------
    def trace_state(self, e: int, face: int, own: bool = True) -> np.ndarray:
        """u0 at the face points of `face` of element e, [n^(d-1), nc]: own side, or the
        neighbour's trace at the same points (own=False)."""
        E = self.scalar._face_eval(face, own=own)
        src = e if own else self.mesh.neighbor(e, face)
        return (E @ self.U0[src].T)

    def face_data(self, e: int, face: int):
        """(own Jacobian 1/2 (A_n(u0-) + lam I), neighbour 1/2 (A_n(u0+) - lam I)),
        each [n^(d-1), nc, nc], and lam [n^(d-1)]."""
        nvec = self.normals[face]
        um, up = self.trace_state(e, face, True), self.trace_state(e, face, False)
        Am, Ap = self.flux.jacobians(um), self.flux.jacobians(up)
        Anm = sum(nvec[d] * Am[d] for d in range(self.dim))
        Anp = sum(nvec[d] * Ap[d] for d in range(self.dim))
        lam = np.maximum(self.flux.speed(um, nvec), self.flux.speed(up, nvec))
        I = np.eye(self.nc)
        own = 0.5 * (Anm + lam[:, None, None] * I)
        nbr = 0.5 * (Anp - lam[:, None, None] * I)
        return own, nbr, lam

    # -- blocks --------------------------------------------------------------------
    def _derivative_mats(self):
        """K_d: the weak derivative in direction d, (D^T W on d, G^T W elsewhere)."""
        b = self.basis
        GtW, DtW = b.G.T @ b.W, b.D.T @ b.W
        return [_kron_all([DtW if t == d else GtW for t in range(self.dim - 1, -1, -1)])
                for d in range(self.dim)]

    def _volume(self, e: int) -> np.ndarray:
        b = self.basis
        G = _kron_all([b.G] * self.dim)
        K = self._derivative_mats()
        A = self.flux.jacobians(self.U0[e].T)                 # each [nloc, nc, nc]
        out = np.zeros((self.bs, self.bs))
        nl = self.nloc
        for c in range(self.nc):
            for c2 in range(self.nc):
                blk = sum(K[d] @ np.diag(self.hf * A[d][:, c, c2]) @ G for d in range(self.dim))
                out[c * nl:(c + 1) * nl, c2 * nl:(c2 + 1) * nl] = blk
        return out

    def element_block(self, e: int) -> np.ndarray:
        """Full diagonal block S_e (n_c n^d square)."""
        M = np.kron(np.eye(self.nc), self.scalar.mass_block(e))
        S = M - self.dt * self._volume(e)
        wf = self.scalar._face_weights()
        nl = self.nloc
        for face in range(2 * self.dim):
            E = self.scalar._face_eval(face, own=True)
            own, _, _ = self.face_data(e, face)
            for c in range(self.nc):
                for c2 in range(self.nc):
                    S[c * nl:(c + 1) * nl, c2 * nl:(c2 + 1) * nl] += \
                        self.dt * self.hf * E.T @ np.diag(wf * own[:, c, c2]) @ E
        return S

    def neighbour_block(self, e: int, face: int) -> np.ndarray:
        wf = self.scalar._face_weights()
        E = self.scalar._face_eval(face, own=True)
        En = self.scalar._face_eval(face, own=False)
        _, nbr, _ = self.face_data(e, face)
        out = np.zeros((self.bs, self.bs))
        nl = self.nloc
        for c in range(self.nc):
            for c2 in range(self.nc):
                out[c * nl:(c + 1) * nl, c2 * nl:(c2 + 1) * nl] = \
                    self.dt * self.hf * E.T @ np.diag(wf * nbr[:, c, c2]) @ En
        return out

    def small_block(self, e: int, c: int) -> np.ndarray:
        """The component-c diagonal sub-block of S_e (the 'small' block)."""
        S = self.element_block(e)
        return S[c * self.nloc:(c + 1) * self.nloc, c * self.nloc:(c + 1) * self.nloc]

    def full_block_ksvd(self, e: int):
        """Rank-2 Kronecker approximation of the full block S_e (2D; Sec. 5.3: A_k of
        size n_c (p+1), B_k of size p+1).  Reading: with the DOF order (component, y, x)
        the A factor acts on the (component, y) index c n + j and B on x, so the
        rearrangement is the one of ksvd with m1 = n1 = n_c n, m2 = n2 = n.  Returns
        (sigma_all, [A_1, A_2], [B_1, B_2])."""
        assert self.dim == 2
        from .ksvd import ksvd
        m = self.nc * self.n
        return ksvd(self.element_block(e), m, m, self.n, self.n, 2)

    def full_block_ksvd_3d(self, e: int):
        """Nested Kronecker approximation A_1 (x) (B_1 (x) C_1 + B_2 (x) C_2) of the full 3D
        block S_e (Sec. 4.3 applied to the n_c n^3 block).  Reading: with the DOF order
        (component, z, y, x) the first-stage factor A_1 acts on the (component, z) index
        c n + k (size n_c n) and D_1 on (y, x); the second stage splits D_1 as in 2D.
        Returns dict(s1, A1, D1, s2, B1, C1, B2, C2, P)."""
        assert self.dim == 3
        from .ksvd import ksvd
        n, m = self.n, self.nc * self.n
        s1, (A1,), (D1,) = ksvd(self.element_block(e), m, m, n * n, n * n, 1)
        s2, (B1, B2), (C1, C2) = ksvd(D1, n, n, n, n, 2)
        P = np.kron(A1, np.kron(B1, C1) + np.kron(B2, C2))
        return dict(s1=s1, A1=A1, D1=D1, s2=s2, B1=B1, C1=C1, B2=B2, C2=C2, P=P)

    def global_matrix(self) -> sp.csr_matrix:
        bs = self.bs
        rows, cols, vals = [], [], []
        for e in range(self.mesh.num_elem):
            blocks = [(e, self.element_block(e))]
            blocks += [(self.mesh.neighbor(e, f), self.neighbour_block(e, f))
                       for f in range(2 * self.dim)]
            for col, B in blocks:
                r, c = np.nonzero(B)
                rows.append(e * bs + r)
                cols.append(col * bs + c)
                vals.append(B[r, c])
        return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                             shape=(self.ndof, self.ndof))

    def mass_matrix(self) -> sp.csr_matrix:
        blocks = [np.kron(np.eye(self.nc), self.scalar.mass_block(e))
                  for e in range(self.mesh.num_elem)]
        return sp.csr_matrix(sp.block_diag(blocks))

    # -- nonlinear residual (for the finite-difference pin) --------------------------
    def residual(self, U: np.ndarray, lam_frozen) -> np.ndarray:
        """dt times the nonlinear DG residual R(U) = -(volume) + (faces) of the
        conservation law at the nodal state U [E, nc, n^d], with the LLF flux and the
        dissipation coefficients lam_frozen[e][face]; J = dR/dU at U0."""
        K = self._derivative_mats()
        wf = self.scalar._face_weights()
        U = U.reshape(self.mesh.num_elem, self.nc, self.nloc)
        out = np.zeros_like(U)
        for e in range(self.mesh.num_elem):
            F = self.flux.flux(U[e].T)                         # each [nloc, nc]
            out[e] -= sum(K[d] @ (self.hf * F[d]) for d in range(self.dim)).T
            for face in range(2 * self.dim):
                nvec = self.normals[face]
                E = self.scalar._face_eval(face, own=True)
                En = self.scalar._face_eval(face, own=False)
                um = E @ U[e].T
                up = En @ U[self.mesh.neighbor(e, face)].T
                fm, fp = self.flux.flux(um), self.flux.flux(up)
                Fn = 0.5 * sum(nvec[d] * (fm[d] + fp[d]) for d in range(self.dim)) + \
                    0.5 * lam_frozen[e][face][:, None] * (um - up)
                out[e] += self.hf * (E.T @ (wf[:, None] * Fn)).T
        return self.dt * out.reshape(-1)


class _ZeroVelocity:
    """A zero scalar velocity, only to reuse AdvectionDG's basis and face matrices."""

    def __init__(self, dim: int):
        self.dim = dim
        self.a0 = np.zeros(dim)
        self.n_modes = 0
        self.amp = np.zeros((dim, 0))
        self.kvec = np.zeros((dim, 0, dim))
        self.phase = np.zeros((dim, 0))


def vortex_system(nel, h, n, dt, state_fn, gamma: float = 1.4) -> LinearizedSystemDG:
    """The Euler system linearised around state_fn (conserved variables at points
    [..., d]) sampled at the nodes of a periodic mesh of nel elements of width h (2D:
    4 components; 3D: 5)."""
    mesh = PeriodicMesh(nel, h)
    flux = EulerFlux(gamma) if mesh.dim == 2 else Euler3DFlux(gamma)
    n_loc = n ** mesh.dim
    sysdg = LinearizedSystemDG(mesh, n, dt, flux, np.zeros((mesh.num_elem, flux.nc, n_loc)))
    U0 = np.empty((mesh.num_elem, flux.nc, n_loc))
    for e in range(mesh.num_elem):
        U0[e] = state_fn(sysdg.scalar.volume_points(e)).T
    sysdg.U0 = U0
    return sysdg
