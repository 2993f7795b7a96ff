"""Host-side logic of the C ABI that needs no GPU: workspace sizing, argument
validation and the network's parameter count (no kernel is launched)."""
import ctypes as C

import numpy as np
import pytest

import synthetic


@pytest.fixture(scope="module")
def L():
    from paper_1704_04549_gb300 import _lib
    from paper_1704_04549_gb300 import build
    build.build()
    _lib.load()
    return _lib


def _problem(L, dim=2, n=8, nel=(4, 4), h=1.0, dt=0.05, nrhs=1, isolated=False, mu=0):
    """A tpp_problem on host arrays (the sizing and validation calls read no array)."""
    from paper_1704_04549_gb300 import mesh
    E = int(np.prod(nel)) if len(nel) else 0
    nbr = (mesh.isolated_nbr(E, dim) if isolated or dim not in (2, 3) or min(nel, default=0) < 1
           else mesh.periodic_nbr(nel))
    keep = dict(nbr=np.ascontiguousarray(nbr, dtype=np.int32))
    P = L.Problem()
    P.dim, P.n, P.num_elem, P.nrhs, P.mu = dim, n, E, nrhs, mu
    P.h, P.dt = h, dt
    P.nbr = keep["nbr"].ctypes.data_as(C.c_void_p)
    return P, keep


def test_network_parameter_count(L):
    lib = L.load()
    # 513 -> 512 -> 512 -> 512 -> 1024 with biases: the 1.31M parameters of the n = 16 network
    assert lib.tpp_mlp_num_params(16) == 513 * 512 + 512 + 2 * (512 * 512 + 512) + 512 * 1024 + 1024
    assert lib.tpp_mlp_num_params(16) == 1313792
    assert lib.tpp_mlp_num_params(2) == 9 * 512 + 512 + 2 * (512 * 512 + 512) + 512 * 16 + 16
    assert lib.tpp_mlp_num_params(0) == -1 and lib.tpp_mlp_num_params(33) == -1
    small, big = lib.tpp_mlp_workspace_bytes(16, 64), lib.tpp_mlp_workspace_bytes(16, 4096)
    assert 0 < small < big
    assert lib.tpp_mlp_workspace_bytes(1, 64) == 0 and lib.tpp_mlp_workspace_bytes(16, 0) == 0


def test_workspace_sizing_and_validation(L):
    lib = L.load()
    P, keep = _problem(L)
    base = lib.tpp_workspace_bytes(C.byref(P), 30, 0)
    assert base > 0
    mixed = lib.tpp_workspace_bytes(C.byref(P), 30, L.TPP_FEAT_MIXED)
    learned = lib.tpp_workspace_bytes(C.byref(P), 30, L.TPP_FEAT_LEARNED)
    assert mixed > base and learned > base
    assert lib.tpp_workspace_bytes(C.byref(P), 10, 0) < base       # smaller Krylov basis
    P2, keep2 = _problem(L, nel=(8, 8))
    assert lib.tpp_workspace_bytes(C.byref(P2), 30, 0) > base      # more elements
    for bad in (dict(n=0), dict(n=33), dict(dim=4), dict(nel=(0, 4)), dict(h=0.0),
                dict(dt=-1.0), dict(dim=3, n=17, nel=(2, 2, 2)), dict(nrhs=0)):
        Pb, kb = _problem(L, **bad)
        assert lib.tpp_workspace_bytes(C.byref(Pb), 30, 0) == 0, bad
    assert lib.tpp_workspace_bytes(C.byref(P), 0, 0) == 0
    assert lib.tpp_workspace_bytes(C.byref(P), 64, 0) == 0
    # right-hand sides per element scale the vectors, not the factors
    Pc, kc = _problem(L, nel=(5, 1), nrhs=3, isolated=True)
    P1, k1 = _problem(L, nel=(5, 1), nrhs=1, isolated=True)
    assert lib.tpp_workspace_bytes(C.byref(Pc), 30, 0) > lib.tpp_workspace_bytes(C.byref(P1), 30, 0)
    # one of the velocity arrays without the other
    v = np.zeros(2 * 16 * 64)
    P.vel_nodes = v.ctypes.data_as(C.c_void_p)
    assert lib.tpp_workspace_bytes(C.byref(P), 30, 0) == 0


def test_over_integration_sizing_and_validation(L):
    """mu = 0 and mu = n are the collocated rule; n < mu <= 32 over-integrates in 2D
    (explicit cores of size min(n^2, 2 mu + 2), operator coefficients at mu^2 points)."""
    lib = L.load()
    base = lib.tpp_workspace_bytes(C.byref(_problem(L)[0]), 30, 0)
    assert lib.tpp_workspace_bytes(C.byref(_problem(L, mu=8)[0]), 30, 0) == base
    P12, k12 = _problem(L, mu=12)
    assert lib.tpp_workspace_bytes(C.byref(P12), 30, 0) > base
    for bad in (dict(mu=5), dict(mu=33), dict(mu=-1), dict(dim=3, n=4, nel=(2, 2, 2), mu=6)):
        Pb, kb = _problem(L, **bad)
        assert lib.tpp_workspace_bytes(C.byref(Pb), 30, 0) == 0, bad


def test_invalid_arguments_are_reported_without_a_device(L):
    lib = L.load()
    P, keep = _problem(L)
    st = lib.tpp_create(None, C.byref(P), 30, 0, None, 0, None)
    assert st == 1 and b"NULL" in lib.tpp_last_error()
    ctx = C.c_void_p()
    st = lib.tpp_create(C.byref(ctx), C.byref(P), 30, 0, None, 0, None)
    assert st != 0 and not ctx.value
    assert lib.tpp_core_size(None) == -1 and lib.tpp_num_dofs(None) == -1
    net = C.c_void_p()
    assert lib.tpp_mlp_create(C.byref(net), 1, 8, None, 0, None) == 1
    assert not net.value


def test_invalid_neighbour_table_is_rejected_before_any_device_work(L):
    """A NULL neighbour table is refused by tpp_create (the workspace check and the
    table's range check come before any kernel)."""
    lib = L.load()
    P, keep = _problem(L)
    P.nbr = None
    ctx = C.c_void_p()
    assert lib.tpp_create(C.byref(ctx), C.byref(P), 30, 0, None, 0, None) == 1
    assert b"nbr" in lib.tpp_last_error() and not ctx.value


@pytest.mark.parametrize("nel", [(4, 3), (3, 2, 5)])
def test_periodic_mesh_arrays(nel):
    """Neighbour table: the element across face f sees e across its opposite face; face
    values: both sides of every face carry opposite a.n; volume values are the field at
    the normalised node positions (x fastest)."""
    from paper_1704_04549_gb300 import mesh
    dim = len(nel)
    nbr = mesh.periodic_nbr(nel)
    E = int(np.prod(nel))
    assert nbr.shape == (E, 2 * dim) and nbr.min() >= 0 and nbr.max() < E
    for f in range(2 * dim):
        assert np.array_equal(nbr[nbr[:, f], f ^ 1], np.arange(E))
    x = np.array([0.2, 0.7, 0.9])
    vel = synthetic.fourier_velocity(1705, dim)
    vn, fn = mesh.periodic_field(nel, x, vel)
    n = len(x)
    assert vn.shape == (dim, E * n ** dim) and fn.shape == (E, 2 * dim, n ** (dim - 1))
    for f in range(2 * dim):
        assert np.array_equal(fn[nbr[:, f], f ^ 1], -fn[:, f])
    # node (i, j[, k]) of element (ex, ey[, ez]) sits at ((ex + x_i) / N_x, ...)
    e = E - 1
    c = np.unravel_index(e, tuple(reversed(nel)))[::-1]
    q = 1 + n * 2 if dim == 2 else 1 + n * 2 + n * n * 0
    ijk = (1, 2) if dim == 2 else (1, 2, 0)
    X = np.array([(c[d] + x[ijk[d]]) / nel[d] for d in range(dim)])
    assert np.allclose(vn[:, e * n ** dim + q], synthetic.velocity_values(vel, X), rtol=0,
                       atol=1e-14)


def test_isolated_element_arrays():
    """Isolated elements: no neighbours; the lower and upper face values are the field
    at the faces of the element's sampled span, with the outward sign."""
    from paper_1704_04549_gb300 import mesh
    cen = np.array([[0.3, 0.6], [0.9, 0.1]])
    x = np.array([0.25, 0.75])
    vel = synthetic.fourier_velocity(7, 2)
    nbr = mesh.isolated_nbr(2, 2)
    assert (nbr == -1).all()
    vn, fn = mesh.isolated_field(cen, x, vel, span=0.1)
    # +x face of element 1, tangential node 0: (0.9 + 0.05, 0.1 + 0.1 (0.25 - 0.5))
    a = synthetic.velocity_values(vel, np.array([0.95, 0.1 - 0.025]))
    assert abs(fn[1, 1, 0] - a[0]) <= 1e-15
    a = synthetic.velocity_values(vel, np.array([0.3 + 0.1 * (0.75 - 0.5), 0.55]))
    assert abs(fn[0, 2, 1] + a[1]) <= 1e-15        # -y face: outward normal -e_y


def test_system_problem_validation(L):
    """tpp_sys_workspace_bytes rejects what tpp_create_system would (no kernel runs)."""
    lib = L.load()
    from paper_1704_04549_gb300 import mesh
    nbr = np.ascontiguousarray(mesh.periodic_nbr((3, 3)), dtype=np.int32)
    state = np.ones(9 * 4 * 16)

    def problem(**kw):
        P = L.SysProblem()
        P.dim, P.n, P.num_elem, P.nc, P.flux = 2, 4, 9, 4, L.TPP_FLUX_EULER
        P.gamma, P.h, P.dt = 1.4, 1.0, 0.1
        P.state = state.ctypes.data_as(C.c_void_p)
        P.nbr = nbr.ctypes.data_as(C.c_void_p)
        for k, v in kw.items():
            setattr(P, k, v)
        return P
    good = lib.tpp_sys_workspace_bytes(C.byref(problem()), 30, 0)
    assert good > 0
    scalar, _ = _problem(L, n=4, nel=(36,), isolated=True)
    assert good > lib.tpp_workspace_bytes(C.byref(scalar), 30, 0)   # + the coupling arrays
    for bad in (dict(dim=3), dict(nc=5), dict(flux=0), dict(gamma=1.0), dict(n=0), dict(h=0.0),
                dict(state=None)):
        assert lib.tpp_sys_workspace_bytes(C.byref(problem(**bad)), 30, 0) == 0, bad
    assert lib.tpp_sys_workspace_bytes(C.byref(problem()), 4, 0) == 0        # max_restart >= 5
    assert lib.tpp_sys_workspace_bytes(C.byref(problem()), 30, L.TPP_FEAT_MIXED) == 0
    assert b"TPP_FEAT" in lib.tpp_last_error()
    # 3D: five components, n <= 12, and a Krylov basis large enough for the diagonal
    # coefficient scratch, (max_restart + 1) n >= dim (n + 2)
    nbr3 = np.ascontiguousarray(mesh.periodic_nbr((2, 2, 2)), dtype=np.int32)
    p3 = dict(dim=3, nc=5, num_elem=8, nbr=nbr3.ctypes.data_as(C.c_void_p))
    g3 = lib.tpp_sys_workspace_bytes(C.byref(problem(**p3)), 30, 0)
    assert g3 > 0
    for bad in (dict(nc=4), dict(n=13)):
        assert lib.tpp_sys_workspace_bytes(C.byref(problem(**{**p3, **bad})), 30, 0) == 0, bad
    assert lib.tpp_sys_workspace_bytes(C.byref(problem(**{**p3, 'n': 1})), 7, 0) == 0   # 8 < 9
    assert lib.tpp_sys_workspace_bytes(C.byref(problem(**{**p3, 'n': 1})), 8, 0) > 0
    assert lib.tpp_sys_workspace_bytes(C.byref(problem(**{**p3, 'n': 12})), 30, 0) > g3
    # full blocks: Kronecker factors 2D (n <= 16) and 3D (nested); exact LU 3D n <= 6
    FULL, BJ = L.TPP_FEAT_FULL_BLOCKS, L.TPP_FEAT_BLOCK_JACOBI
    assert lib.tpp_sys_workspace_bytes(C.byref(problem()), 30, FULL) > good
    assert lib.tpp_sys_workspace_bytes(C.byref(problem()), 30, FULL | BJ) > \
        lib.tpp_sys_workspace_bytes(C.byref(problem()), 30, FULL)
    assert lib.tpp_sys_workspace_bytes(C.byref(problem(n=17)), 30, FULL) == 0
    assert lib.tpp_sys_workspace_bytes(C.byref(problem()), 30, FULL | L.TPP_FEAT_TWO_SIDED) == 0
    assert lib.tpp_sys_workspace_bytes(C.byref(problem(**p3)), 30, FULL) > 0
    assert lib.tpp_sys_workspace_bytes(C.byref(problem(**p3)), 30, FULL | L.TPP_FEAT_TWO_SIDED) == 0
    assert lib.tpp_sys_workspace_bytes(C.byref(problem(**p3)), 30, FULL | BJ) > 0
    assert lib.tpp_sys_workspace_bytes(C.byref(problem(**{**p3, 'n': 7})), 30, FULL | BJ) == 0


def test_batch_and_metric_argument_checks(L):
    """The batched GMRES checks its options before touching a context, and the metric
    terms entry point rejects NULL arguments; neither needs a device."""
    lib = L.load()
    o = L.BatchOpts()
    o.restart, o.max_iters, o.rtol, o.prec = 20, 100, 1e-8, L.TPP_FP64
    dummy = (C.c_void_p * 1)(None)
    assert lib.tpp_batch_workspace_bytes(dummy, 1, C.byref(o)) == 0          # NULL context
    assert b"NULL" in lib.tpp_last_error()
    for field, val in (("restart", 0), ("restart", 32), ("max_iters", 0), ("rtol", 0.0),
                       ("prec", 7)):
        ob = L.BatchOpts()
        C.pointer(ob)[0] = o
        setattr(ob, field, val)
        assert lib.tpp_batch_workspace_bytes(dummy, 1, C.byref(ob)) == 0, field
    om = L.BatchOpts()
    C.pointer(om)[0] = o
    om.prec, om.max_outer, om.inner_rtol = L.TPP_FP32, 0, 1e-4
    assert lib.tpp_batch_workspace_bytes(dummy, 1, C.byref(om)) == 0
    assert lib.tpp_set_metric_terms(None, None, None, None, 0.1, None) == 1  # NULL context


def test_f32_shifts_feature_validation(L):
    """TPP_FEAT_F32_SHIFTS: with TPP_FEAT_MIXED and the one-sided form only; the 2 n^3
    FP64 shifted inverses per element are then not reserved."""
    lib = L.load()
    P, _keep = _problem(L, n=16, nel=(4, 4))
    MIX, F32S = L.TPP_FEAT_MIXED, L.TPP_FEAT_F32_SHIFTS
    full = lib.tpp_workspace_bytes(C.byref(P), 30, MIX)
    lean = lib.tpp_workspace_bytes(C.byref(P), 30, MIX | F32S)
    assert 0 < lean and full - lean >= 16 * 2 * 16 ** 3 * 8
    for bad in (F32S, F32S | MIX | L.TPP_FEAT_TWO_SIDED, F32S | MIX | L.TPP_FEAT_BF16,
                F32S | MIX | L.TPP_FEAT_TIME, F32S | MIX | L.TPP_FEAT_LEARNED):
        assert lib.tpp_workspace_bytes(C.byref(P), 30, bad) == 0, bad
    assert b"TPP_FEAT_F32_SHIFTS" in lib.tpp_last_error()
    P17, _k17 = _problem(L, n=17, nel=(2, 2))
    assert lib.tpp_workspace_bytes(C.byref(P17), 30, MIX | F32S) == 0
    P3, _k3 = _problem(L, dim=3, n=6, nel=(2, 2, 2))
    assert lib.tpp_workspace_bytes(C.byref(P3), 30, MIX | F32S) > 0
