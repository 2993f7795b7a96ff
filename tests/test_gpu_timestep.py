"""GPU: time integration (backward Euler, Alexander's DIRK3 with KSVD-preconditioned
GMRES stages, explicit RK4) against the oracle's integrators on the same mesh."""
import numpy as np
import pytest
import torch

import synthetic
from oracle import timestep as T
from oracle.dg import AdvectionDG, PeriodicMesh
from paper_1704_04549_gb300 import (TPP_FEAT_TIME, TPP_TS_BACKWARD_EULER, TPP_TS_DIRK3,
                                    TPP_TS_RK4)
from tests.gpu_util import make_pair, rel, to_dev, to_host

pytestmark = pytest.mark.gpu

SCHEMES = {"be": (TPP_TS_BACKWARD_EULER, T.backward_euler),
           "dirk3": (TPP_TS_DIRK3, T.dirk3), "rk4": (TPP_TS_RK4, T.rk4)}


@pytest.mark.parametrize("name,dt,steps", [("be", 0.05, 4), ("dirk3", 0.05, 4),
                                           ("rk4", 0.002, 25)])
@pytest.mark.parametrize("dim,n,nel", [(2, 6, (4, 4)), (3, 4, (2, 3, 2))])
def test_integrators_match_oracle(name, dt, steps, dim, n, nel):
    """Same scheme, same dt and steps on the same periodic mesh: the GPU solution
    equals the oracle's (direct stage solves) to the GMRES tolerance; 1^T M u is
    conserved."""
    scheme, ref = SCHEMES[name]
    vel = synthetic.fourier_velocity(1705, dim)
    ctx, dg = make_pair(n, nel, 0.05, vel, features=TPP_FEAT_TIME, h=1.0)
    m, J = T.spatial_operator(dg)
    u0 = synthetic.rhs(1716, dg.ndof)
    u = to_dev(u0)
    rep = ctx.tpp_time_integrate(u, scheme, dt, steps, rtol=1e-12)
    u_ref = ref(m, J, u0, dt, steps)
    uh = to_host(u)
    assert rep["steps"] == steps
    assert rel(uh, u_ref) <= 1e-9, rel(uh, u_ref)
    assert abs(m @ uh - m @ u0) <= 1e-9 * np.abs(m * u0).sum()
    if name != "rk4":
        assert rep["solves"] == steps * (3 if name == "dirk3" else 1)
        assert rep["max_true_rel_res"] <= 1e-12 and rep["builds"] == 1


def test_dirk3_rebuild_each_step_and_third_order():
    """Rebuilding the factors before every step (the paper's setting) gives the same
    solution; DIRK3's error against the exact semi-discrete solution falls by about
    2^3 when dt is halved (on the GPU path)."""
    vel = synthetic.fourier_velocity(1705, 2, kmax=1)
    ctx, dg = make_pair(5, (3, 3), 0.05, vel, features=TPP_FEAT_TIME, h=1.0)
    m, J = T.spatial_operator(dg)
    u0 = synthetic.rhs(1717, dg.ndof)
    t_end = 0.2
    ex = T.exact(m, J, u0, t_end)
    errs = []
    for k in (1, 2):
        u = to_dev(u0)
        h = 0.05 / k
        rep = ctx.tpp_time_integrate(u, TPP_TS_DIRK3, h, int(round(t_end / h)), rtol=1e-13)
        errs.append(np.linalg.norm(to_host(u) - ex))
    rate = np.log2(errs[0] / errs[1])
    assert abs(rate - 3.0) <= 0.3, (errs, rate)
    u1, u2 = to_dev(u0), to_dev(u0)
    ctx.tpp_time_integrate(u1, TPP_TS_DIRK3, 0.05, 3, rtol=1e-13)
    rep = ctx.tpp_time_integrate(u2, TPP_TS_DIRK3, 0.05, 3, rebuild_each_step=True, rtol=1e-13)
    assert rep["builds"] == 3
    assert torch.equal(u1, u2)
