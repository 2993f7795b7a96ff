"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This module only draws random numbers, fixes workload sizes and evaluates the
drawn velocity fields at given points; it holds none of the method's arithmetic
(no basis, quadrature, operator, factorisation or solver).  The oracle evaluates
the field parameters with its own code; the CUDA path receives field values at
its nodes from ``velocity_values``.

Velocity fields are described by parameters, not values: component ``c`` is

    a_c(x) = a0[c] + sum_m amp[c, m] * cos(2*pi * kvec[c, m, :] . x + phase[c, m])

with integer wavevectors, so every field is periodic on the unit cube.

Random-Fourier recipe (default, divergence-free like the paper's advection
fields of Sec. 5.1): mode m draws a scalar amplitude A_m ~ U(-1, 1), a
wavevector k_m with components uniform in {1..kmax} and a phase
phi_m ~ U(0, 2 pi), and contributes A_m e_m cos(2 pi k_m . x + phi_m) with
e_m a unit vector perpendicular to k_m (2D: (k_y, -k_x)/|k|; 3D: a random
unit vector orthogonalised against k_m), so div a = 0 exactly.  Every
component of one mode shares its wavevector and phase.

``solenoidal=False`` draws an independent amplitude, wavevector and phase per
component instead (not divergence-free).  A separable field (each component
depends only on its own coordinate, the case in which Eq. adv-kron-cart makes
the diagonal block an exact two-term Kronecker sum) keeps only the c-th
wavevector component of component c.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Velocity:
    dim: int
    a0: np.ndarray                       # [dim]
    amp: np.ndarray                      # [dim, M]
    kvec: np.ndarray                     # [dim, M, dim] int32
    phase: np.ndarray                    # [dim, M]

    @property
    def n_modes(self) -> int:
        return int(self.amp.shape[1])


def constant_velocity(a) -> Velocity:
    a = np.asarray(a, dtype=np.float64)
    d = a.shape[0]
    return Velocity(d, a.copy(), np.zeros((d, 0)), np.zeros((d, 0, d), np.int32),
                    np.zeros((d, 0)))


def fourier_velocity(seed: int, dim: int, n_modes: int = 8, kmax: int = 4,
                     a0=None, separable: bool = False, solenoidal: bool = True) -> Velocity:
    rng = np.random.Generator(np.random.PCG64(seed))
    a0 = np.zeros(dim) if a0 is None else np.asarray(a0, dtype=np.float64)
    if separable or not solenoidal:
        amp = rng.uniform(-1.0, 1.0, size=(dim, n_modes))
        kvec = rng.integers(1, kmax + 1, size=(dim, n_modes, dim)).astype(np.int32)
        phase = rng.uniform(0.0, 2.0 * np.pi, size=(dim, n_modes))
        if separable:
            for c in range(dim):
                for d in range(dim):
                    if d != c:
                        kvec[c, :, d] = 0
        return Velocity(dim, a0, amp, kvec, phase)
    A = rng.uniform(-1.0, 1.0, size=n_modes)
    k = rng.integers(1, kmax + 1, size=(n_modes, dim)).astype(np.int32)
    phi = rng.uniform(0.0, 2.0 * np.pi, size=n_modes)
    amp = np.zeros((dim, n_modes))
    for m in range(n_modes):
        km = k[m].astype(np.float64)
        if dim == 2:
            e = np.array([km[1], -km[0]])
        else:
            e = rng.standard_normal(3)
            e -= (e @ km) / (km @ km) * km
        amp[:, m] = A[m] * e / np.linalg.norm(e)
    kvec = np.broadcast_to(k[None], (dim, n_modes, dim)).astype(np.int32).copy()
    phase = np.broadcast_to(phi[None], (dim, n_modes)).copy()
    return Velocity(dim, a0, amp, kvec, phase)


def velocity_values(vel: Velocity, X: np.ndarray) -> np.ndarray:
    """Values of the field at points X[..., dim] of the unit cube (the series above);
    returns [..., dim] float64."""
    X = np.asarray(X, dtype=np.float64)
    out = np.empty(X.shape[:-1] + (vel.dim,))
    for c in range(vel.dim):
        val = np.full(X.shape[:-1], float(vel.a0[c]))
        for m in range(vel.n_modes):
            k = vel.kvec[c, m].astype(np.float64)
            val += vel.amp[c, m] * np.cos(2.0 * np.pi * (X @ k) + vel.phase[c, m])
        out[..., c] = val
    return out


@dataclass
class ElementMaps:
    """Geometry of E elements of width h for the mass-matrix workloads: element e maps
    the reference cube [0, 1]^dim by
      bilinear:  the multilinear interpolation of its corners, each corner of the
                 reference cube moved by h * eps * (a U(-1, 1) vector);
      curved:    x = h (xi + eps sum_d s_d sin(2 pi xi_{d+1} + phi_{e,d}) e_d), a smooth
                 non-polynomial map (indices cyclic);
      affine:    x = h xi.
    ``jacobian(e, X)`` is |det dx/dxi| at reference points X[..., dim]."""
    kind: str
    dim: int
    h: float
    eps: float
    corners: np.ndarray      # [E, 2^dim, dim] corner displacements (bilinear)
    phase: np.ndarray        # [E, dim] (curved)

    @property
    def num_elem(self) -> int:
        return int(self.phase.shape[0])

    def jacobian(self, e: int, X: np.ndarray) -> np.ndarray:
        X = np.asarray(X, dtype=np.float64)
        d = self.dim
        Jm = np.zeros(X.shape[:-1] + (d, d))
        if self.kind == "affine":
            Jm[...] = np.eye(d)
        elif self.kind == "curved":
            Jm[...] = np.eye(d)
            for c in range(d):
                nxt = (c + 1) % d
                Jm[..., c, nxt] += self.eps * 2 * np.pi * np.cos(
                    2 * np.pi * X[..., nxt] + self.phase[e, c])
        else:
            # x(xi) = sum_corners N_k(xi) (corner_k + h eps delta_k) / h-scaled below
            for k in range(2 ** d):
                bits = [(k >> c) & 1 for c in range(d)]
                corner = np.array(bits, dtype=np.float64) + self.eps * self.corners[e, k]
                for c in range(d):         # derivative of N_k along c
                    dN = np.ones(X.shape[:-1])
                    for q in range(d):
                        f = X[..., q] if bits[q] else 1.0 - X[..., q]
                        if q == c:
                            f = np.ones(X.shape[:-1]) if bits[q] else -np.ones(X.shape[:-1])
                        dN = dN * f
                    Jm[..., :, c] += dN[..., None] * corner
        return np.abs(np.linalg.det(Jm)) * self.h ** d


def element_maps(seed: int, num_elem: int, dim: int, kind: str, h: float = 1.0,
                 eps: float = 0.1) -> ElementMaps:
    rng = np.random.Generator(np.random.PCG64(seed))
    corners = rng.uniform(-1.0, 1.0, size=(num_elem, 2 ** dim, dim))
    phase = rng.uniform(0.0, 2 * np.pi, size=(num_elem, dim))
    return ElementMaps(kind, dim, h, eps, corners, phase)


def rhs(seed: int, ndof: int) -> np.ndarray:
    """Right-hand side b ~ N(0, 1), float64."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal(ndof)


@dataclass
class Workload:
    name: str
    dim: int
    n: int                     # Gauss-Legendre nodes per direction (p + 1)
    nel: tuple                 # elements per direction (periodic)
    dt: float
    velocity: Velocity
    rhs_seed: int
    h: float = 1.0          # unit-square (unit-cube) elements; domain [0, N h]^d

    @property
    def num_elem(self) -> int:
        return int(np.prod(self.nel))

    @property
    def ndof(self) -> int:
        return self.num_elem * self.n ** self.dim

    def b(self) -> np.ndarray:
        return rhs(self.rhs_seed, self.ndof)


def advection_2d_const(n: int = 8, nel: int = 8, dt: float = 0.1) -> Workload:
    """8x8 periodic unit-square quads, p = 7, constant velocity (1, 0.5), dt = 0.1."""
    return Workload(f"adv2d-const-{nel}x{nel}-n{n}", 2, n, (nel, nel), dt,
                    constant_velocity([1.0, 0.5]), rhs_seed=1704)


def advection_2d_fourier(n: int = 16, nel: int = 64, dt: float = 0.05,
                         vel_seed: int = 1705, rhs_seed: int = 1706) -> Workload:
    """64x64 periodic unit-square quads, n = 16 or 31, random-Fourier velocity, dt = 0.05."""
    return Workload(f"adv2d-fourier-{nel}x{nel}-n{n}", 2, n, (nel, nel), dt,
                    fourier_velocity(vel_seed, 2), rhs_seed=rhs_seed)


def advection_3d_fourier(n: int = 11, nel: int = 16, dt: float = 0.05,
                         vel_seed: int = 1707, rhs_seed: int = 1708) -> Workload:
    """16^3 periodic unit-cube hexes, n = 11, random-Fourier velocity, dt = 0.05."""
    return Workload(f"adv3d-fourier-{nel}^3-n{n}", 3, n, (nel, nel, nel), dt,
                    fourier_velocity(vel_seed, 3), rhs_seed=rhs_seed)


@dataclass
class DegreeGroup:
    """Elements of one (dimension, n) group of a mixed-degree batch."""
    dim: int
    n: int
    centres: np.ndarray        # [E_g, dim], uniform in the unit cube
    ids: np.ndarray            # positions of these elements in the whole batch
    rhs_seed: int              # b ~ N(0, 1) of shape [E_g][R][n^dim] from this seed


def mixed_degree_batch(seed: int = 1709, e2d: int = 20000, e3d: int = 2000,
                       p2d=(4, 30), p3d=(3, 12)):
    """Mixed-degree batch of isolated elements: degrees p ~ U{p2d} (2D) and U{p3d}
    (3D), element centres uniform in [0, 1]^d, grouped by (dim, n = p + 1) in
    increasing n.  Returns the list of groups (element ids refer to the draw order,
    2D elements first)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    p2 = rng.integers(p2d[0], p2d[1] + 1, size=e2d)
    c2 = rng.random((e2d, 2))
    p3 = rng.integers(p3d[0], p3d[1] + 1, size=e3d)
    c3 = rng.random((e3d, 3))
    groups = []
    for dim, ps, cs, off in ((2, p2, c2, 0), (3, p3, c3, e2d)):
        for p in np.unique(ps):
            sel = np.nonzero(ps == p)[0]
            groups.append(DegreeGroup(dim, int(p) + 1, cs[sel], sel + off,
                                      rhs_seed=seed * 1000 + dim * 100 + int(p)))
    return groups


# ---------------------------------------------------------------------------
# Linearisation state of the 2D Euler workload (Sec. 5.3, the moving isentropic vortex at
# t = 0): conserved variables (rho, rho u, rho v, rho E) at points X [..., 2].
VORTEX = dict(gamma=1.4, mach=0.5, u_inf=1.0, theta=float(np.arctan(0.5)), eps=0.3, rc=1.5,
              x0=5.0, y0=5.0, rho_inf=1.0)


def euler_vortex_state(X: np.ndarray, params: dict = VORTEX) -> np.ndarray:
    """The vortex of Sec. 5.3 with the paper's parameters (M = 0.5, u_inf = 1, theta =
    atan(1/2), eps = 0.3, r_c = 1.5, centre (5, 5)); p_inf = rho_inf u_inf^2 / (gamma M^2)
    (free-stream Mach number M).  Returns [..., 4] conserved variables."""
    P = params
    g = P["gamma"]
    X = np.asarray(X, dtype=np.float64)
    dx, dy = X[..., 0] - P["x0"], X[..., 1] - P["y0"]
    f = (1.0 - dx * dx - dy * dy) / P["rc"] ** 2
    s = P["eps"] / (2.0 * np.pi * P["rc"]) * np.exp(0.5 * f)
    u = P["u_inf"] * (np.cos(P["theta"]) - s * dy)
    v = P["u_inf"] * (np.sin(P["theta"]) + s * dx)
    base = 1.0 - P["eps"] ** 2 * (g - 1.0) * P["mach"] ** 2 / (8.0 * np.pi ** 2) * np.exp(f)
    rho = P["rho_inf"] * base ** (1.0 / (g - 1.0))
    p_inf = P["rho_inf"] * P["u_inf"] ** 2 / (g * P["mach"] ** 2)
    p = p_inf * base ** (g / (g - 1.0))
    E = p / ((g - 1.0) * rho) + 0.5 * (u * u + v * v)
    return np.stack([rho, rho * u, rho * v, rho * E], axis=-1)


# ---------------------------------------------------------------------------
# Curved (non-affine) elements: a smooth periodic warp of the periodic square of side L,
#   Phi(X) = X + alpha L sin(2 pi X / L) sin(2 pi Y / L) (1, 1),
# a bijection of the torus onto itself for 2 pi alpha < 1 (det grad Phi =
# 1 + 2 pi alpha sin(2 pi (X + Y) / L) > 0).  Elements are the images of the
# Cartesian cells: x = Phi((c + xi) h).
def periodic_warp(X: np.ndarray, L: float, alpha: float = 0.05):
    """(x = Phi(X) [..., 2], grad Phi [..., 2, 2] with [..., i, j] = d x_i / d X_j)."""
    X = np.asarray(X, dtype=np.float64)
    k = 2.0 * np.pi / L
    sx, sy = np.sin(k * X[..., 0]), np.sin(k * X[..., 1])
    cx, cy = np.cos(k * X[..., 0]), np.cos(k * X[..., 1])
    p = alpha * L * sx * sy
    x = np.stack([X[..., 0] + p, X[..., 1] + p], axis=-1)
    dpx, dpy = alpha * L * k * cx * sy, alpha * L * k * sx * cy
    G = np.empty(X.shape[:-1] + (2, 2))
    G[..., 0, 0] = 1.0 + dpx
    G[..., 0, 1] = dpy
    G[..., 1, 0] = dpx
    G[..., 1, 1] = 1.0 + dpy
    return x, G


def periodic_warp3(X: np.ndarray, L: float, alpha: float = 0.03):
    """3D counterpart of periodic_warp: x = X + alpha L sin(kX) sin(kY) sin(kZ) (1, 1, 1),
    k = 2 pi / L, a smooth map of the periodic cube onto itself.  Returns (x [..., 3],
    grad Phi [..., 3, 3] with [..., i, j] = d x_i / d X_j)."""
    X = np.asarray(X, dtype=np.float64)
    k = 2.0 * np.pi / L
    s = np.sin(k * X)
    c = np.cos(k * X)
    p = alpha * L * s[..., 0] * s[..., 1] * s[..., 2]
    x = X + p[..., None]
    dp = alpha * L * k * np.stack([c[..., 0] * s[..., 1] * s[..., 2],
                                   s[..., 0] * c[..., 1] * s[..., 2],
                                   s[..., 0] * s[..., 1] * c[..., 2]], axis=-1)
    G = np.broadcast_to(np.eye(3), X.shape[:-1] + (3, 3)).copy()
    G += dp[..., None, :]
    return x, G


# Linearisation state of the 3D Euler workload: the initial condition of the periodic
# case of Sec. 5.6 (its exact solution is a travelling wave), density
# rho = 1 + 0.2 sin(2 pi (x + y + z) / L) (L = 2: sin(pi (x + y + z))) advected by the
# uniform velocity (1, -1/2, 1) at uniform pressure 1 (gamma = 1.4).
def euler3d_wave_state(X: np.ndarray, L: float, gamma: float = 1.4) -> np.ndarray:
    """Conserved variables (rho, rho u, rho v, rho w, rho E) [..., 5] at points X [..., 3]."""
    X = np.asarray(X, dtype=np.float64)
    rho = 1.0 + 0.2 * np.sin(2.0 * np.pi * X.sum(-1) / L)
    V = np.array([1.0, -0.5, 1.0])
    p = 1.0
    E = p / ((gamma - 1.0) * rho) + 0.5 * float(V @ V)
    return np.concatenate([rho[..., None], rho[..., None] * V, (rho * E)[..., None]], -1)
