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


def _problem(L, dim=2, n=8, nel=(4, 4), h=1.0, dt=0.05, batch_rhs=0, centres=None):
    vel = synthetic.fourier_velocity(1705, dim if dim in (2, 3) else 2)
    keep = dict(a0=np.ascontiguousarray(vel.a0, dtype=np.float64),
                amp=np.ascontiguousarray(vel.amp, dtype=np.float64).reshape(-1),
                kvec=np.ascontiguousarray(vel.kvec, dtype=np.int32).reshape(-1),
                phase=np.ascontiguousarray(vel.phase, dtype=np.float64).reshape(-1))
    P = L.Problem()
    P.dim, P.n = dim, n
    for d in range(3):
        P.nel[d] = nel[d] if d < len(nel) else 1
    P.h, P.dt, P.n_modes = h, dt, np.asarray(vel.amp).shape[1]
    P.a0 = keep["a0"].ctypes.data_as(C.POINTER(C.c_double))
    P.amp = keep["amp"].ctypes.data_as(C.POINTER(C.c_double))
    P.kvec = keep["kvec"].ctypes.data_as(C.POINTER(C.c_int32))
    P.phase = keep["phase"].ctypes.data_as(C.POINTER(C.c_double))
    P.batch_rhs = batch_rhs
    if centres is not None:
        keep["centres"] = np.ascontiguousarray(centres, dtype=np.float64)
        P.centres = keep["centres"].ctypes.data_as(C.POINTER(C.c_double))
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
                dict(dt=-1.0), dict(dim=3, n=17, nel=(2, 2, 2)), dict(batch_rhs=2)):
        Pb, kb = _problem(L, **bad)
        assert lib.tpp_workspace_bytes(C.byref(Pb), 30, 0) == 0, bad
    assert lib.tpp_workspace_bytes(C.byref(P), 0, 0) == 0
    assert lib.tpp_workspace_bytes(C.byref(P), 64, 0) == 0
    Pc, kc = _problem(L, nel=(5,), batch_rhs=3, centres=np.full((5, 2), 0.5))
    assert lib.tpp_workspace_bytes(C.byref(Pc), 30, 0) > 0


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
