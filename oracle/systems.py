"""Linearised DG operator of a system of conservation laws in 2D (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Sec. 5.3 and Sec. 5.6: for the Euler equations the unknowns have n_c components
(n_c = 4 in 2D: rho, rho u, rho v, rho E, flux of Eq. euler-flux), so the diagonal
blocks of the Jacobian are n_c n^2 x n_c n^2 ("full" blocks); the "small" blocks
are their n_c diagonal n^2 x n^2 sub-blocks, which do not couple the components.

The DG discretisation is the one of oracle/dg.py (collocated Gauss-Legendre nodes,
periodic Cartesian mesh of square elements of width h) applied to every
component, with the local Lax-Friedrichs numerical flux
  F^(u-, u+) . n = 1/2 (F(u-) + F(u+)) . n + 1/2 lam (u- - u+),
  lam = max(|v- . n| + c-, |v+ . n| + c+)
(the generic numerical flux of Sec. 2; the paper does not name the one used for
Euler).  Linearised around a DG state u0 (its nodal values; traces by the face
evaluation matrices) with lam frozen at its value for u0, the residual's
Jacobian has
  volume   -dt sum_d (D^T W (x) G^T W or G^T W (x) D^T W) diag(h A_d[c, c'](u0))
  faces    own:  dt h E^T diag(w_f 1/2 (A_n(u0-)[c, c'] + lam delta_cc')) E
           nbr:  dt h E^T diag(w_f 1/2 (A_n(u0+)[c, c'] - lam delta_cc')) E'
with A_d = dF_d/du and A_n = n_x A_x + n_y A_y for the outward normal n.
S = M - dt J as in oracle/dg.py.  DOF ordering: element, then component, then
node i + n j (x fastest).

Pinned in tests/test_oracle_systems.py: the analytic Euler Jacobians against
finite differences of the flux, the eigenvalues of A_n (v.n - c, v.n, v.n,
v.n + c), the reduction of a one-component linear "system" (flux a u, lam =
|a.n|) to the upwind advection operator of oracle/dg.py, discrete conservation of
every component, and J x against a finite difference of the nonlinear DG residual.
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


class EulerFlux:
    nc = 4

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
    reduction pin against oracle/dg.py)."""
    nc = 1

    def __init__(self, a):
        self.a = np.asarray(a, dtype=np.float64)

    def flux(self, U):
        return self.a[0] * U, self.a[1] * U

    def jacobians(self, U):
        shp = U.shape[:-1] + (1, 1)
        return np.full(shp, self.a[0]), np.full(shp, self.a[1])

    def speed(self, U, nvec):
        return np.full(U.shape[:-1], abs(self.a[0] * nvec[0] + self.a[1] * nvec[1]))


# outward normals of the faces -x, +x, -y, +y
NORMALS = ((-1.0, 0.0), (1.0, 0.0), (0.0, -1.0), (0.0, 1.0))


class LinearizedSystemDG:
    """S = M - dt J of a 2D system linearised around the nodal state U0 [E, nc, n^2]."""

    def __init__(self, mesh: PeriodicMesh, n: int, dt: float, flux, U0: np.ndarray):
        assert mesh.dim == 2
        self.mesh, self.n, self.dt, self.flux = mesh, n, float(dt), flux
        self.nc = flux.nc
        self.scalar = AdvectionDG(mesh, n, dt, _ZeroVelocity())   # basis, face matrices
        self.basis = self.scalar.basis
        self.nloc = n * n
        self.bs = self.nc * self.nloc                 # block size
        self.ndof = mesh.num_elem * self.bs
        self.U0 = np.asarray(U0, dtype=np.float64).reshape(mesh.num_elem, self.nc, self.nloc)

    # -- linearisation data -------------------------------------------------------
    def trace_state(self, e: int, face: int, own: bool = True) -> np.ndarray:
        """u0 at the face points of `face` of element e, [n, nc]: own side, or the
        neighbour's trace at the same points (own=False)."""
        E = self.scalar._face_eval(face, own=own)
        src = e if own else self.mesh.neighbor(e, face)
        return (E @ self.U0[src].T)

    def face_data(self, e: int, face: int):
        """(own Jacobian 1/2 (A_n(u0-) + lam I), neighbour 1/2 (A_n(u0+) - lam I)),
        each [n, nc, nc], and lam [n]."""
        nvec = NORMALS[face]
        um, up = self.trace_state(e, face, True), self.trace_state(e, face, False)
        Axm, Aym = self.flux.jacobians(um)
        Axp, Ayp = self.flux.jacobians(up)
        Anm = nvec[0] * Axm + nvec[1] * Aym
        Anp = nvec[0] * Axp + nvec[1] * Ayp
        lam = np.maximum(self.flux.speed(um, nvec), self.flux.speed(up, nvec))
        I = np.eye(self.nc)
        own = 0.5 * (Anm + lam[:, None, None] * I)
        nbr = 0.5 * (Anp - lam[:, None, None] * I)
        return own, nbr, lam

    # -- blocks --------------------------------------------------------------------
    def _volume(self, e: int) -> np.ndarray:
        b, h = self.basis, self.mesh.h
        GtW, DtW = b.G.T @ b.W, b.D.T @ b.W
        G = _kron_all([b.G, b.G])
        Ax, Ay = self.flux.jacobians(self.U0[e].T)            # [nloc, nc, nc]
        Kx = _kron_all([GtW, DtW])                             # x derivative on the fast index
        Ky = _kron_all([DtW, GtW])
        out = np.zeros((self.bs, self.bs))
        for c in range(self.nc):
            for c2 in range(self.nc):
                blk = Kx @ np.diag(h * Ax[:, c, c2]) @ G + Ky @ np.diag(h * Ay[:, c, c2]) @ G
                out[c * self.nloc:(c + 1) * self.nloc, c2 * self.nloc:(c2 + 1) * self.nloc] = blk
        return out

    def element_block(self, e: int) -> np.ndarray:
        """Full diagonal block S_e (n_c n^2 square)."""
        h = self.mesh.h
        M = np.kron(np.eye(self.nc), self.scalar.mass_block(e))
        S = M - self.dt * self._volume(e)
        wf = self.scalar._face_weights()
        for face in range(4):
            E = self.scalar._face_eval(face, own=True)
            own, _, _ = self.face_data(e, face)
            for c in range(self.nc):
                for c2 in range(self.nc):
                    S[c * self.nloc:(c + 1) * self.nloc, c2 * self.nloc:(c2 + 1) * self.nloc] += \
                        self.dt * h * E.T @ np.diag(wf * own[:, c, c2]) @ E
        return S

    def neighbour_block(self, e: int, face: int) -> np.ndarray:
        h = self.mesh.h
        wf = self.scalar._face_weights()
        E = self.scalar._face_eval(face, own=True)
        En = self.scalar._face_eval(face, own=False)
        _, nbr, _ = self.face_data(e, face)
        out = np.zeros((self.bs, self.bs))
        for c in range(self.nc):
            for c2 in range(self.nc):
                out[c * self.nloc:(c + 1) * self.nloc, c2 * self.nloc:(c2 + 1) * self.nloc] = \
                    self.dt * h * E.T @ np.diag(wf * nbr[:, c, c2]) @ En
        return out

    def small_block(self, e: int, c: int) -> np.ndarray:
        """The component-c diagonal sub-block of S_e (the 'small' block)."""
        S = self.element_block(e)
        return S[c * self.nloc:(c + 1) * self.nloc, c * self.nloc:(c + 1) * self.nloc]

    def global_matrix(self) -> sp.csr_matrix:
        rows = []
        bs = self.bs
        A = sp.lil_matrix((self.ndof, self.ndof))
        for e in range(self.mesh.num_elem):
            A[e * bs:(e + 1) * bs, e * bs:(e + 1) * bs] = self.element_block(e)
            for face in range(4):
                nb = self.mesh.neighbor(e, face)
                blk = self.neighbour_block(e, face)
                cur = A[e * bs:(e + 1) * bs, nb * bs:(nb + 1) * bs].toarray()
                A[e * bs:(e + 1) * bs, nb * bs:(nb + 1) * bs] = cur + blk
        del rows
        return A.tocsr()

    def mass_matrix(self) -> sp.csr_matrix:
        blocks = [np.kron(np.eye(self.nc), self.scalar.mass_block(e))
                  for e in range(self.mesh.num_elem)]
        return sp.block_diag(blocks).tocsr()

    # -- nonlinear residual (for the finite-difference pin) --------------------------
    def residual(self, U: np.ndarray, lam_frozen) -> np.ndarray:
        """dt times the nonlinear DG residual R(U) = -(volume) + (faces) of the
        conservation law at the nodal state U [E, nc, n^2], with the LLF flux and the
        dissipation coefficients lam_frozen[e][face] ([n]); J = dR/dU at U0."""
        b, h = self.basis, self.mesh.h
        GtW, DtW = b.G.T @ b.W, b.D.T @ b.W
        Kx, Ky = _kron_all([GtW, DtW]), _kron_all([DtW, GtW])
        wf = self.scalar._face_weights()
        U = U.reshape(self.mesh.num_elem, self.nc, self.nloc)
        out = np.zeros_like(U)
        for e in range(self.mesh.num_elem):
            F1, F2 = self.flux.flux(U[e].T)                    # [nloc, nc]
            out[e] -= (Kx @ (h * F1) + Ky @ (h * F2)).T
            for face in range(4):
                nvec = NORMALS[face]
                E = self.scalar._face_eval(face, own=True)
                En = self.scalar._face_eval(face, own=False)
                um = E @ U[e].T
                up = En @ U[self.mesh.neighbor(e, face)].T
                f1m, f2m = self.flux.flux(um)
                f1p, f2p = self.flux.flux(up)
                Fn = 0.5 * (nvec[0] * (f1m + f1p) + nvec[1] * (f2m + f2p)) + \
                    0.5 * lam_frozen[e][face][:, None] * (um - up)
                out[e] += h * (E.T @ (wf[:, None] * Fn)).T
        return self.dt * out.reshape(-1)


class _ZeroVelocity:
    """A zero scalar velocity, only to reuse AdvectionDG's basis and face matrices."""
    dim = 2
    a0 = np.zeros(2)
    n_modes = 0
    amp = np.zeros((2, 0))
    kvec = np.zeros((2, 0, 2))
    phase = np.zeros((2, 0))


def vortex_system(nel, h, n, dt, state_fn, gamma: float = 1.4) -> LinearizedSystemDG:
    """The Euler system linearised around state_fn (conserved variables at points
    [..., 2]) sampled at the nodes of an nel[0] x nel[1] periodic mesh of width h."""
    mesh = PeriodicMesh(nel, h)
    sysdg = LinearizedSystemDG(mesh, n, dt, EulerFlux(gamma),
                               np.zeros((mesh.num_elem, 4, n * n)))
    U0 = np.empty((mesh.num_elem, 4, n * n))
    for e in range(mesh.num_elem):
        U0[e] = state_fn(sysdg.scalar.volume_points(e)).T
    sysdg.U0 = U0
    return sysdg
