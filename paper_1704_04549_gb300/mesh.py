"""Problem arrays for libtpp's tpp_problem: connectivity and field values.

Host-side setup of the two element layouts the workloads use (Sec. 3.4: the
library needs a.n at the face nodes, a at the volume nodes and the neighbour
across every face; it evaluates nothing itself):

* ``periodic_nbr`` / ``periodic_field``: N_1 x ... periodic Cartesian elements of width h, element
  e = ex + N_1 (ey + N_2 ez); the field is a function of the normalised point
  x / L (L_d = N_d h), so it is periodic on the mesh for every h.  A face is
  evaluated once, at the coordinates of the element that owns it as its lower
  face, and both sides get opposite values of a.n_outward.
* ``isolated_nbr`` / ``isolated_field``: a batch of block-diagonal systems, element e the cube of
  width h centred at centres[e] in the unit domain, the field sampled over
  `span` around the centre; no neighbours (nbr = -1).

Node coordinates use the Gauss-Legendre nodes of the context (read from the
library), face nodes are ordered by their tangential indices (x, y, z order,
first fastest) and faces -x, +x, -y, +y (, -z, +z).
"""
from __future__ import annotations

import numpy as np

import synthetic


def _tangential(dim: int, axis: int):
    return [d for d in range(dim) if d != axis]


def _coords(nel):
    E = int(np.prod(nel))
    coords, rest = [], np.arange(E)
    for N in nel:
        coords.append(rest % N)
        rest //= N
    return E, coords


def periodic_nbr(nel) -> np.ndarray:
    """Neighbour table [E, 2 dim] (int32) of the periodic Cartesian mesh of nel elements."""
    nel = tuple(int(v) for v in nel)
    dim = len(nel)
    E, coords = _coords(nel)
    strides = np.cumprod((1,) + nel[:-1])

    def shifted(d, s):
        c = [cc.copy() for cc in coords]
        c[d] = (c[d] + s) % nel[d]
        return sum(ci * st for ci, st in zip(c, strides))

    nbr = np.empty((E, 2 * dim), dtype=np.int32)
    for d in range(dim):
        nbr[:, 2 * d] = shifted(d, -1)
        nbr[:, 2 * d + 1] = shifted(d, +1)
    return nbr


def isolated_nbr(num_elem: int, dim: int) -> np.ndarray:
    """Neighbour table of isolated elements: every face uncoupled (-1)."""
    return np.full((num_elem, 2 * dim), -1, dtype=np.int32)


def periodic_field(nel, x: np.ndarray, velocity):
    """(vel_nodes [dim, E n^dim], vel_face_normal [E, 2 dim, n^(dim-1)]) of the periodic
    mesh of nel elements with the 1D nodes x on [0, 1]."""
    nel = tuple(int(v) for v in nel)
    dim, n = len(nel), len(x)
    E, coords = _coords(nel)
    nbr = periodic_nbr(nel)
    # volume nodes: normalised point ((e_d + x_i) / N_d), node index i + n j (+ n^2 k)
    grids = np.meshgrid(*([x] * dim), indexing="ij")          # grids[d][i, j, (k)]
    X = np.empty((E,) + (n,) * dim + (dim,))
    for d in range(dim):
        shape = (E,) + (1,) * dim
        X[..., d] = (coords[d].reshape(shape) + grids[d][None]) / nel[d]
    # flatten with x fastest
    X = np.transpose(X, (0,) + tuple(range(dim, 0, -1)) + (dim + 1,)).reshape(E, n ** dim, dim)
    vel_nodes = np.ascontiguousarray(
        np.moveaxis(synthetic.velocity_values(velocity, X), -1, 0).reshape(dim, -1))
    # faces: value of a_d at each element's lower d-face (owner), then both sides
    nfl = n ** (dim - 1)
    tg = np.meshgrid(*([x] * (dim - 1)), indexing="ij") if dim > 1 else []
    fn = np.empty((E, 2 * dim, nfl))
    for d in range(dim):
        tang = _tangential(dim, d)
        P = np.empty((E,) + (n,) * (dim - 1) + (dim,))
        P[..., d] = (coords[d] / nel[d]).reshape((E,) + (1,) * (dim - 1))
        for a, t in enumerate(tang):
            P[..., t] = (coords[t].reshape((E,) + (1,) * (dim - 1)) + tg[a][None]) / nel[t]
        P = np.transpose(P, (0,) + tuple(range(dim - 1, 0, -1)) + (dim,)).reshape(E, nfl, dim)
        a_low = synthetic.velocity_values(velocity, P)[..., d]      # a_d on e's lower face
        fn[:, 2 * d, :] = -a_low                                    # outward -e_d
        fn[:, 2 * d + 1, :] = a_low[nbr[:, 2 * d + 1]]              # the +d neighbour's lower face
    return vel_nodes, np.ascontiguousarray(fn)


def isolated_field(centres: np.ndarray, x: np.ndarray, velocity, span: float):
    """(vel_nodes, vel_face_normal) of isolated elements centred at centres [E, dim]
    whose field is sampled over `span` (coordinates of the unit domain)."""
    centres = np.asarray(centres, dtype=np.float64)
    E, dim = centres.shape
    n = len(x)
    grids = np.meshgrid(*([x] * dim), indexing="ij")
    X = np.empty((E,) + (n,) * dim + (dim,))
    for d in range(dim):
        X[..., d] = centres[:, d].reshape((E,) + (1,) * dim) + span * (grids[d][None] - 0.5)
    X = np.transpose(X, (0,) + tuple(range(dim, 0, -1)) + (dim + 1,)).reshape(E, n ** dim, dim)
    vel_nodes = np.ascontiguousarray(
        np.moveaxis(synthetic.velocity_values(velocity, X), -1, 0).reshape(dim, -1))
    nfl = n ** (dim - 1)
    tg = np.meshgrid(*([x] * (dim - 1)), indexing="ij") if dim > 1 else []
    fn = np.empty((E, 2 * dim, nfl))
    for d in range(dim):
        tang = _tangential(dim, d)
        for up in (0, 1):
            P = np.empty((E,) + (n,) * (dim - 1) + (dim,))
            P[..., d] = (centres[:, d] + span * (up - 0.5)).reshape((E,) + (1,) * (dim - 1))
            for a, t in enumerate(tang):
                P[..., t] = centres[:, t].reshape((E,) + (1,) * (dim - 1)) + \
                    span * (tg[a][None] - 0.5)
            P = np.transpose(P, (0,) + tuple(range(dim - 1, 0, -1)) + (dim,)).reshape(E, nfl, dim)
            a = synthetic.velocity_values(velocity, P)[..., d]
            fn[:, 2 * d + up, :] = a if up else -a
    return vel_nodes, np.ascontiguousarray(fn)


def warped_metric_terms(nel, h: float, x: np.ndarray, velocity, warp):
    """Metric terms of tpp_set_metric_terms for the 2D periodic mesh of nel = (N, N)
    square cells of width h mapped by `warp` (X -> (Phi(X), grad Phi(X)), a bijection of
    the periodic square of side L = N h, e.g. synthetic.periodic_warp): element e is
    x = Phi((c + xi) h) and J_T = h grad Phi.  x: the context's quadrature points on
    [0, 1] (tpp_gauss_legendre).  Returns (jdet [E][q^2], flux [2][E][q^2],
    flux_face [E][4][q]); the velocity is evaluated at the physical point divided by L.
    A face's geometry is computed from the element that owns it as its lower face, so
    the two sides get opposite scaled normal velocities."""
    nel = tuple(int(v) for v in nel)
    assert len(nel) == 2 and nel[0] == nel[1]
    L = nel[0] * h
    q = len(x)
    E, (cx, cy) = _coords(nel)
    # volume points, a + q b with x fastest
    xi_x = np.tile(x, q)
    xi_y = np.repeat(x, q)
    X = np.stack([(cx[:, None] + xi_x[None, :]) * h, (cy[:, None] + xi_y[None, :]) * h], -1)
    phys, G = warp(X)
    J = h * G
    det = J[..., 0, 0] * J[..., 1, 1] - J[..., 0, 1] * J[..., 1, 0]
    a = synthetic.velocity_values(velocity, phys / L)
    # |J| J^-1 a = adj(J) a
    fx = J[..., 1, 1] * a[..., 0] - J[..., 0, 1] * a[..., 1]
    fy = -J[..., 1, 0] * a[..., 0] + J[..., 0, 0] * a[..., 1]
    flux = np.stack([fx, fy], 0)
    ff = np.empty((E, 4, q))
    normals = ((-1.0, 0.0), (1.0, 0.0), (0.0, -1.0), (0.0, 1.0))
    for f in range(4):
        d, side = divmod(f, 2)
        XF = np.empty((E, q, 2))
        own = (cx if d == 0 else cy) + side
        tang = cy if d == 0 else cx
        XF[..., d] = own[:, None] * h
        XF[..., 1 - d] = (tang[:, None] + x[None, :]) * h
        pf, GF = warp(XF)
        JF = h * GF
        # |J| J^-T N = adj(J)^T N
        nx, ny = normals[f]
        sx = JF[..., 1, 1] * nx - JF[..., 1, 0] * ny
        sy = -JF[..., 0, 1] * nx + JF[..., 0, 0] * ny
        af = synthetic.velocity_values(velocity, pf / L)
        ff[:, f, :] = af[..., 0] * sx + af[..., 1] * sy
    return det, flux, ff
