"""Parity of the CUDA viscous chain (common solution, gradients, BR1-type
common viscous fluxes, isothermal moving walls, viscous mortar procedure of
Sec. 3.2) with the FP64 oracle, and Taylor-Couette accuracy (Sec. 4.2)."""
import math

import numpy as np
import pytest

from helpers import rel_err, small_rotor
from ssd_inputs import fields, meshes
from ssd_inputs.workloads import FlowParams, build_workload

pytestmark = pytest.mark.gpu

TOL64 = (1e-12, 1e-12)  # FP64 residuals against the extended-precision oracle; states against the FP64 oracle
TOL32_RESIDUAL = (5e-5, 5e-4)
TOL32_STATE = (1e-5, 1e-5)


@pytest.fixture(scope="module")
def ssd():
    import paper_1503_02198_gb300 as pkg
    pkg.build()
    return pkg


def _check(a, b, tol):
    l2 = np.sqrt(((a - b) ** 2).sum(axis=(0, 2, 3)) / (b ** 2).sum(axis=(0, 2, 3)))
    mx = rel_err(a, b)
    assert (l2 <= tol[0]).all() and (mx <= tol[1]).all(), (l2, mx)


def _couette_params(omega=1.0, mach=0.1, re=10.0):
    gamma, Tw = 1.4, 1.0
    Rgas = (omega / mach) ** 2 / (gamma * Tw)
    return FlowParams(gamma=gamma, Rgas=Rgas, mu=omega / re, prandtl=0.72, omega=omega, viscous=1, T_wall=Tw)


@pytest.mark.parametrize("N", [3, 4])
@pytest.mark.parametrize("precision", [0, 1])
def test_couette_residual(ssd, oracle_mod, N, precision):
    m = meshes.couette_mesh(2, 12, 2, 16, phi_out=0.05)
    prm = _couette_params()
    s, o = ssd.Solver(m, N - 1, prm, precision=precision), oracle_mod.Oracle(m, N, prm)
    Q = o.state_from(lambda x, y: fields.random_smooth_state(x, y, seed=N, amp=0.05, u0=0.2, v0=-0.1,
                                                             p0=prm.Rgas))
    s.sd_set_state(Q)
    s.sd_set_time(0.43)
    _check(s.sd_residual(), (o.extended() if precision == 0 else o).residual(Q, 0.43), TOL64 if precision == 0 else TOL32_RESIDUAL)


@pytest.mark.parametrize("precision", [0, 1])
def test_viscous_rotor_residual(ssd, oracle_mod, precision):
    m = small_rotor(shift_R=0.05)
    prm = FlowParams(omega=0.7, viscous=1, mu=0.02, Rgas=1.0, prandtl=0.72)
    s, o = ssd.Solver(m, 3, prm, precision=precision), oracle_mod.Oracle(m, 4, prm)
    Q = o.state_from(lambda x, y: fields.random_smooth_state(x, y, seed=2, amp=0.2, scale=3.0))
    s.sd_set_state(Q)
    s.sd_set_time(1.9)
    _check(s.sd_residual(), (o.extended() if precision == 0 else o).residual(Q, 1.9), TOL64 if precision == 0 else TOL32_RESIDUAL)


@pytest.mark.parametrize("precision", [0, 1])
def test_couette_config_steps(ssd, oracle_mod, precision):
    # the Taylor-Couette configuration itself: 4x32 rotating + 4x40 stationary
    # cells, N = 3, Mach 0.1, Re = 10, omega = 0.5, 200 SSP-RK3 steps
    w = build_workload("couette_n3")
    s, o = ssd.Solver(w.mesh, w.N - 1, w.params, precision=precision), oracle_mod.Oracle(w.mesh, w.N, w.params)
    p0 = w.params.Rgas * w.params.T_wall
    Q = o.state_from(lambda x, y: fields.uniform(x, y, rho=1.0, p=p0))
    s.sd_set_state(Q)
    s.sd_step(w.cfl_dt, w.steps)
    s.sd_sync()
    q_ref, t_ref = o.step(Q, 0.0, w.cfl_dt, w.steps)
    assert abs(s.sd_get_time() - t_ref) < 1e-13
    _check(s.sd_get_state(), q_ref, TOL64 if precision == 0 else TOL32_STATE)


def test_couette_accuracy_order(ssd):
    # Sec. 4.2: steady Taylor-Couette flow; the error of u against the exact
    # circumferential velocity falls at about order N (paper: 3.1 at N = 3).
    # As in the paper, each mesh is run until its error stops changing.
    prm = _couette_params(omega=1.0)
    k = prm.mu * prm.gamma * prm.Rgas / ((prm.gamma - 1) * prm.prandtl)
    ex = fields.CouetteExact(1.0, 1.0, 2.0, prm.mu, k, prm.Rgas, prm.T_wall)
    N = 3
    errs = []
    for scale in (1, 2):
        m = meshes.couette_mesh(3 * scale, 16 * scale, 3 * scale, 20 * scale)
        s = ssd.Solver(m, N - 1, prm)
        xy = s.sd_sp_coords(0.0)
        s.sd_set_state(np.ascontiguousarray(np.moveaxis(ex.state(xy[..., 0], xy[..., 1]), -1, 1)))
        h = 0.5 / (3 * scale)
        c = math.sqrt(prm.gamma * prm.Rgas * prm.T_wall)
        dt = 0.2 * h / ((c + 1.0) * N * N)
        chunk = int(math.ceil(1.0 / dt))
        prev = None
        for _ in range(16):
            s.sd_step(dt, chunk)
            s.sd_sync()
            t = s.sd_get_time()
            Q = s.sd_get_state()
            xy = s.sd_sp_coords(t)
            x, y = xy[..., 0], xy[..., 1]
            r = np.hypot(x, y)
            err = np.sqrt(np.mean((Q[:, 1] / Q[:, 0] + ex.v(r) * y / r) ** 2))
            if prev is not None and abs(err - prev) < 1e-3 * err:
                break
            prev = err
        errs.append(err)
    order = math.log2(errs[0] / errs[1])
    assert order > N - 0.5, (errs, order)


@pytest.mark.parametrize("precision", [0, 1])
def test_couette_rk54_steps(ssd, oracle_mod, precision):
    w = build_workload("couette_n3")
    prm = w.params
    prm.rk_stages = 5
    s, o = ssd.Solver(w.mesh, w.N - 1, prm, precision=precision), oracle_mod.Oracle(w.mesh, w.N, prm)
    Q = o.state_from(lambda x, y: fields.uniform(x, y, rho=1.0, p=prm.Rgas * prm.T_wall))
    s.sd_set_state(Q)
    s.sd_step(w.cfl_dt, 20)
    s.sd_sync()
    q_ref, _ = o.step(Q, 0.0, w.cfl_dt, 20, rk_stages=5)
    _check(s.sd_get_state(), q_ref, TOL64 if precision == 0 else TOL32_STATE)
