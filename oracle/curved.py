"""DG discretisation of linear advection on curved (non-affine) 2D elements (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The general-geometry form of Sec. 3.2 (Eq. mass-kron and adv-kron with a full
element Jacobian J_T): element e is the image x = Phi((c + xi) h) of the Cartesian
cell c of width h under a smooth map Phi of the periodic square of side L (the map
and its gradient are inputs, synthetic.periodic_warp).  With the reference
Jacobian J = dx/dxi = h grad Phi at a quadrature point, |J| = det J, and the
contravariant flux velocity F~ = |J| J^-1 a, the weak form gives, point by point
(quadrature points and weights of the mu-point rule, tensor product):
  mass     M   = G^T diag(w |J|) G                  (G = G1 (x) G1)
  volume   J_v = Dx^T diag(w F~_x) G + Dy^T diag(w F~_y) G
                                                    (Dx = G1 (x) D1, Dy = D1 (x) G1)
  faces    own  E^T diag(w_f max(a . s, 0)) E,  neighbour  E^T diag(w_f min(a . s, 0)) E'
           with the scaled normal s = |J| J^-T N^ (N^ the reference outward normal),
and S = M - dt J_v + dt (faces), as in oracle/dg.py (upwind flux).  The geometry of
a face point is computed from the element that owns the face as its lower face, so
the two sides of a face see s and -s exactly.  The velocity is a(x / L) with the
field of oracle/dg.py (periodic on the square).

CurvedAdvectionDG3D is the same construction on hexahedra (synthetic.periodic_warp3), for
which the CUDA path is not built yet.

Pinned in tests/test_oracle_curved.py (both classes): the identity map reproduces oracle/dg.py
(collocated and over-integrated), the warp's gradient against finite differences,
discrete conservation 1^T (S - M) = 0 for the warped map, opposite scaled normal
velocities on the two sides of every face, the mass of the whole domain equal to the
area L^2 and a single element's area converging spectrally, and the free-stream
identity (constant velocity, u = 1: volume and face terms cancel by the divergence
theorem) reached as the quadrature is refined.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .basis import Basis1D
from .dg import PeriodicMesh, velocity_eval

NHAT = ((-1.0, 0.0), (1.0, 0.0), (0.0, -1.0), (0.0, 1.0))   # faces -x, +x, -y, +y


class CurvedAdvectionDG:
    """S = M + dt A on the warped periodic mesh (2D)."""

    def __init__(self, mesh: PeriodicMesh, n: int, dt: float, vel, warp, mu: int | None = None):
        assert mesh.dim == 2
        self.mesh, self.n, self.dt, self.vel, self.warp = mesh, n, float(dt), vel, warp
        self.dim = 2
        self.basis = Basis1D(n, mu)
        self.mu = self.basis.mu
        self.L = mesh.nel[0] * mesh.h
        assert mesh.nel[0] == mesh.nel[1], "square periodic domain"
        self.nloc = n * n
        self.ndof = mesh.num_elem * self.nloc

    def velocity(self, x):
        return velocity_eval(self.vel, np.asarray(x) / self.L)

    # -- geometry at points ---------------------------------------------------------
    def volume_geometry(self, e: int):
        """(|J|, F~ [q, 2]) at the quadrature points (index a + mu b, x fastest)."""
        b, h = self.basis, self.mesh.h
        cx, cy = self.mesh.coords(e)
        Xg, Yg = np.meshgrid((cx + b.x) * h, (cy + b.x) * h, indexing="xy")
        X = np.stack([Xg, Yg], -1).reshape(-1, 2)
        x, G = self.warp(X)
        J = h * G
        det = J[:, 0, 0] * J[:, 1, 1] - J[:, 0, 1] * J[:, 1, 0]
        a = self.velocity(x)
        Ft = np.einsum("qij,qj->qi", np.linalg.inv(J), a) * det[:, None]
        return det, Ft

    def face_an(self, e: int, face: int) -> np.ndarray:
        """a . (|J| J^-T N^) at the face points of `face` (tangential index fastest),
        geometry from the owner of the face (the element for which it is the lower one)."""
        b, h = self.basis, self.mesh.h
        d, side = divmod(face, 2)
        c = list(self.mesh.coords(e))
        owner = c[d] + side                               # not wrapped: X stays continuous
        t = 1 - d
        X = np.empty((self.mu, 2))
        X[:, d] = owner * h
        X[:, t] = (c[t] + b.x) * h
        x, G = self.warp(X)
        J = h * G
        det = J[:, 0, 0] * J[:, 1, 1] - J[:, 0, 1] * J[:, 1, 0]
        s = np.einsum("qji,j->qi", np.linalg.inv(J), np.array(NHAT[face])) * det[:, None]
        return np.einsum("qi,qi->q", self.velocity(x), s)

    # -- blocks ---------------------------------------------------------------------
    def _G(self):
        b = self.basis
        return np.kron(b.G, b.G), np.kron(b.G, b.D), np.kron(b.D, b.G)

    def mass_block(self, e: int) -> np.ndarray:
        b = self.basis
        G, _, _ = self._G()
        det, _ = self.volume_geometry(e)
        w = np.kron(b.w, b.w)
        return G.T @ np.diag(w * det) @ G

    def volume_jacobian_block(self, e: int) -> np.ndarray:
        b = self.basis
        G, Dx, Dy = self._G()
        _, Ft = self.volume_geometry(e)
        w = np.kron(b.w, b.w)
        return Dx.T @ np.diag(w * Ft[:, 0]) @ G + Dy.T @ np.diag(w * Ft[:, 1]) @ G

    def _face_eval(self, face: int, own: bool = True) -> np.ndarray:
        b = self.basis
        d, side = divmod(face, 2)
        if not own:
            side = 1 - side
        lvec = (b.l1 if side == 1 else b.l0)[None, :]
        return np.kron(lvec, b.G) if d == 1 else np.kron(b.G, lvec)

    def face_blocks(self, e: int):
        wf = self.basis.w
        Fdiag = np.zeros((self.nloc, self.nloc))
        nbrs = {}
        for face in range(4):
            an = self.face_an(e, face)
            E, En = self._face_eval(face, True), self._face_eval(face, False)
            Fdiag += E.T @ np.diag(wf * np.maximum(an, 0.0)) @ E
            nbrs[face] = (self.mesh.neighbor(e, face), E.T @ np.diag(wf * np.minimum(an, 0.0)) @ En)
        return Fdiag, nbrs

    def element_block(self, e: int) -> np.ndarray:
        Fdiag, _ = self.face_blocks(e)
        return self.mass_block(e) - self.dt * self.volume_jacobian_block(e) + self.dt * Fdiag

    def global_matrix(self) -> sp.csr_matrix:
        nl = self.nloc
        rows, cols, vals = [], [], []
        for e in range(self.mesh.num_elem):
            Fdiag, nbrs = self.face_blocks(e)
            blocks = [(e, self.mass_block(e) - self.dt * self.volume_jacobian_block(e)
                       + self.dt * Fdiag)]
            blocks += [(nb, self.dt * B) for nb, B in nbrs.values()]
            for col, B in blocks:
                r, c = np.nonzero(B)
                rows.append(e * nl + r)
                cols.append(col * nl + c)
                vals.append(B[r, c])
        return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                             shape=(self.ndof, self.ndof))

    def mass_matrix(self) -> sp.csr_matrix:
        return sp.block_diag([self.mass_block(e) for e in range(self.mesh.num_elem)]).tocsr()


class CurvedAdvectionDG3D:
    """The same mapped-element discretisation on hexahedra (3D): element e is the image of
    the Cartesian cell c under the warp Phi of the periodic cube (synthetic.periodic_warp3),
    J = h grad Phi at the mu^3 quadrature points (x fastest), the contravariant velocity
    |J| J^-1 a, faces with the scaled normal |J| J^-T N^ computed from the element that owns
    the face as its lower face.  mass G^T diag(w |J|) G, volume sum_d D_d^T diag(w F~_d) G,
    upwind faces, S = M - dt J_v + dt (faces)."""

    def __init__(self, mesh: PeriodicMesh, n: int, dt: float, vel, warp, mu: int | None = None):
        assert mesh.dim == 3
        self.mesh, self.n, self.dt, self.vel, self.warp = mesh, n, float(dt), vel, warp
        self.dim = 3
        self.basis = Basis1D(n, mu)
        self.mu = self.basis.mu
        self.L = np.array([N * mesh.h for N in mesh.nel], dtype=np.float64)
        self.nloc = n ** 3
        self.ndof = mesh.num_elem * self.nloc

    def velocity(self, x):
        return velocity_eval(self.vel, np.asarray(x) / self.L)

    def _grid3(self, c):
        """Reference points of cell c at the mu^3 quadrature points, x fastest."""
        xs = self.basis.x
        Z, Y, X = np.meshgrid(xs, xs, xs, indexing="ij")
        h = self.mesh.h
        return np.stack([(c[0] + X) * h, (c[1] + Y) * h, (c[2] + Z) * h], -1).reshape(-1, 3)

    def volume_geometry(self, e: int):
        x, G = self.warp(self._grid3(self.mesh.coords(e)))
        J = self.mesh.h * G
        det = np.linalg.det(J)
        Ft = np.einsum("qij,qj->qi", np.linalg.inv(J), self.velocity(x)) * det[:, None]
        return det, Ft

    def face_an(self, e: int, face: int) -> np.ndarray:
        """a . (|J| J^-T N^) at the mu^2 points of `face` (the two tangential directions in
        increasing order, the lower one fastest), geometry from the face's owner."""
        d, side = divmod(face, 2)
        c = list(self.mesh.coords(e))
        tang = [t for t in range(3) if t != d]
        xs, h = self.basis.x, self.mesh.h
        B, A = np.meshgrid(xs, xs, indexing="ij")        # A: fast tangential, B: slow
        X = np.empty(A.shape + (3,))
        X[..., d] = (c[d] + side) * h                    # not wrapped: X stays continuous
        X[..., tang[0]] = (c[tang[0]] + A) * h
        X[..., tang[1]] = (c[tang[1]] + B) * h
        x, G = self.warp(X.reshape(-1, 3))
        J = h * G
        det = np.linalg.det(J)
        N = np.zeros(3)
        N[d] = 1.0 if side == 1 else -1.0
        s = np.einsum("qji,j->qi", np.linalg.inv(J), N) * det[:, None]
        return np.einsum("qi,qi->q", self.velocity(x), s)

    def _mats(self):
        b = self.basis
        G = np.kron(b.G, np.kron(b.G, b.G))
        D = [np.kron(b.G, np.kron(b.G, b.D)),              # x derivative (x fastest)
             np.kron(b.G, np.kron(b.D, b.G)),
             np.kron(b.D, np.kron(b.G, b.G))]
        w = np.kron(b.w, np.kron(b.w, b.w))
        return G, D, w

    def _face_eval(self, face: int, own: bool = True) -> np.ndarray:
        b = self.basis
        d, side = divmod(face, 2)
        if not own:
            side = 1 - side
        lvec = (b.l1 if side == 1 else b.l0)[None, :]
        mats = [lvec if t == d else b.G for t in (2, 1, 0)]   # slowest direction first
        return np.kron(mats[0], np.kron(mats[1], mats[2]))

    def mass_block(self, e: int) -> np.ndarray:
        G, _, w = self._mats()
        det, _ = self.volume_geometry(e)
        return G.T @ np.diag(w * det) @ G

    def volume_jacobian_block(self, e: int) -> np.ndarray:
        G, D, w = self._mats()
        _, Ft = self.volume_geometry(e)
        return sum(D[k].T @ np.diag(w * Ft[:, k]) @ G for k in range(3))

    def face_blocks(self, e: int):
        wf = np.kron(self.basis.w, self.basis.w)
        Fdiag = np.zeros((self.nloc, self.nloc))
        nbrs = {}
        for face in range(6):
            an = self.face_an(e, face)
            E, En = self._face_eval(face, True), self._face_eval(face, False)
            Fdiag += E.T @ np.diag(wf * np.maximum(an, 0.0)) @ E
            nbrs[face] = (self.mesh.neighbor(e, face), E.T @ np.diag(wf * np.minimum(an, 0.0)) @ En)
        return Fdiag, nbrs

    def element_block(self, e: int) -> np.ndarray:
        Fdiag, _ = self.face_blocks(e)
        return self.mass_block(e) - self.dt * self.volume_jacobian_block(e) + self.dt * Fdiag

    def global_matrix(self) -> sp.csr_matrix:
        nl = self.nloc
        rows, cols, vals = [], [], []
        for e in range(self.mesh.num_elem):
            Fdiag, nbrs = self.face_blocks(e)
            blocks = [(e, self.mass_block(e) - self.dt * self.volume_jacobian_block(e)
                       + self.dt * Fdiag)]
            blocks += [(nb, self.dt * B) for nb, B in nbrs.values()]
            for col, B in blocks:
                r, c = np.nonzero(B)
                rows.append(e * nl + r)
                cols.append(col * nl + c)
                vals.append(B[r, c])
        return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                             shape=(self.ndof, self.ndof))

    def mass_matrix(self) -> sp.csr_matrix:
        return sp.block_diag([self.mass_block(e) for e in range(self.mesh.num_elem)]).tocsr()

