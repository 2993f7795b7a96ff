"""GPU parity: 1D tables and the sum-factorised operator vs the oracle."""
import numpy as np
import pytest

import synthetic
from oracle.basis import Basis1D
from tests.gpu_util import make_pair, rel, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [1, 2, 3, 8, 16, 31, 32])
def test_tables_match_oracle(n):
    ctx, _ = make_pair(n, (2, 2), 0.1, synthetic.constant_velocity([1.0, 0.5]))
    v = ctx.views()
    b = Basis1D(n)
    assert np.allclose(to_host(v["gl_x"]), b.x, rtol=0, atol=2e-16)
    assert np.allclose(to_host(v["gl_w"]), b.w, rtol=1e-12, atol=0)
    D = to_host(v["D"])
    assert np.abs(D - b.D).max() <= 1e-12 * max(1.0, np.abs(b.D).max())


CASES = [
    (1, (3, 5), 0.1, "const"),
    (2, (4, 3), 0.2, "fourier"),
    (5, (3, 5), 0.05, "fourier"),      # ragged mesh
    (8, (8, 8), 0.1, "const"),         # 8x8 periodic, p = 7, constant (1, 0.5), dt = 0.1
    (8, (4, 4), 0.1, "fourier"),
    (16, (3, 3), 0.05, "fourier"),
    (31, (2, 2), 0.05, "fourier"),
]


@pytest.mark.parametrize("n,nel,dt,field", CASES)
def test_operator_matches_assembled_matrix(n, nel, dt, field):
    vel = (synthetic.constant_velocity([1.0, 0.5]) if field == "const"
           else synthetic.fourier_velocity(1705, 2))
    ctx, dg = make_pair(n, nel, dt, vel)
    S = dg.global_matrix()
    x = synthetic.rhs(7, dg.ndof)
    y = to_host(ctx.dg_apply_sumfact(to_dev(x)))
    y_ref = S @ x
    # FP64 reduction-order differences: relative 1e-12 (norm) / 1e-11 (max entry)
    assert rel(y, y_ref) <= 1e-12
    assert np.abs(y - y_ref).max() <= 1e-11 * np.abs(y_ref).max()


def test_operator_full_size_sampled_elements():
    """64 x 64 unit-square quads, n = 16: sampled element rows vs the oracle's block rows."""
    n, nel = 16, (64, 64)
    vel = synthetic.fourier_velocity(1705, 2)
    ctx, dg = make_pair(n, nel, 0.05, vel, h=1.0)
    x = synthetic.rhs(1706, dg.ndof)
    y = to_host(ctx.dg_apply_sumfact(to_dev(x)))
    nl = dg.nloc
    for e in [0, 63, 64 * 37 + 11, 4095]:
        Fd, nbrs = dg.face_blocks(e)
        ye = (dg.mass_block(e) - dg.dt * dg.volume_jacobian_block(e) + dg.dt * Fd) @ x[e * nl:(e + 1) * nl]
        for face, (nb, Fn) in nbrs.items():
            ye += dg.dt * Fn @ x[nb * nl:(nb + 1) * nl]
        assert rel(y[e * nl:(e + 1) * nl], ye) <= 1e-12


def test_operator_conservation_and_constants_full_size():
    n, nel = 31, (64, 64)
    ctx, dg = make_pair(n, nel, 0.05, synthetic.constant_velocity([1.0, 0.5]))
    one = np.ones(dg.ndof)
    y = to_host(ctx.dg_apply_sumfact(to_dev(one)))
    w = dg.basis.w
    M1 = np.tile(dg.mesh.h ** 2 * np.outer(w, w).reshape(-1), dg.mesh.num_elem)
    # A 1 = 0 is reached by cancellation of terms of size |S| 1: tolerance
    # relative to the largest absolute row sum of one element's block row
    Fd, nbrs = dg.face_blocks(0)
    absrow = np.abs(dg.mass_block(0)) + dg.dt * (np.abs(dg.volume_jacobian_block(0)) + np.abs(Fd))
    scale = (absrow.sum(axis=1) + sum(dg.dt * np.abs(F).sum(axis=1) for _, F in nbrs.values())).max()
    assert np.abs(y - M1).max() <= 1e-14 * scale
