"""The C-ABI library loads and exports every entry point include/tpp.h declares.

No compute call is made (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "tpp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set()
    for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*([A-Za-z_][A-Za-z0-9_]*)\s*\(",
                         src, flags=re.M):
        names.add(m.group(1))
    names.discard("TPP_H")
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1704_04549_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_parses():
    names = declared_functions()
    for must in ["tpp_create", "tpp_build_factors", "tpp_apply_inverse", "dg_apply_sumfact",
                 "gmres_solve", "tpp_workspace_bytes", "tpp_last_error"]:
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_python_binding_declares_the_same_names(lib):
    from paper_1704_04549_gb300 import _lib
    assert set(_lib.EXPORTS) == set(declared_functions())


def test_workspace_query_validates_without_gpu(lib):
    from paper_1704_04549_gb300 import _lib
    L = _lib.load()
    P = _lib.Problem()
    P.dim, P.n, P.num_elem, P.nrhs, P.h, P.dt = 2, 8, 64, 1, 1 / 8, 0.1
    nb = L.tpp_workspace_bytes(ctypes.byref(P), 30, 0)
    assert nb > 31 * 4096 * 8
    P.n = 33
    assert L.tpp_workspace_bytes(ctypes.byref(P), 30, 0) == 0
    P.n = 8
    assert L.tpp_workspace_bytes(ctypes.byref(P), 0, 0) == 0


def test_create_fails_loudly_without_device(lib):
    """On a machine without a GPU, creating a context must fail, never fall back."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1704_04549_gb300 import _lib
    L = _lib.load()
    from paper_1704_04549_gb300 import mesh
    nbr = mesh.periodic_nbr((4, 4))
    P = _lib.Problem()
    P.dim, P.n, P.num_elem, P.nrhs, P.h, P.dt = 2, 4, 16, 1, 1 / 4, 0.1
    P.nbr = nbr.ctypes.data_as(ctypes.c_void_p)
    ctx = ctypes.c_void_p()
    buf = ctypes.create_string_buffer(1 << 16)
    st = L.tpp_create(ctypes.byref(ctx), ctypes.byref(P), 30, 0, ctypes.cast(buf, ctypes.c_void_p),
                      1 << 16, None)
    assert st != 0
