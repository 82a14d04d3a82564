"""Parity of the CUDA path with the FP64 oracle on 12-node cubic cells and the
boundary conditions of Sec. 4's elliptic-cylinder case (slip walls, Dirichlet
inlet, fixed-pressure outlet, isothermal no-slip rotating body) and stirred
tank (adiabatic rotating blades, baffles), through the C ABI.  Tolerances as
in test_gpu_parity."""
import numpy as np
import pytest

from helpers import rel_err
from ssd_inputs import fields, meshes
from ssd_inputs.meshes import BC_ADIABATIC, BC_INLET, BC_OUTLET, BC_SLIP
from ssd_inputs.workloads import FlowParams, build_workload, ellipse_params, tank_params

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


def _small_ellipse():
    return meshes.ellipse_mesh(n_theta=32, n_inner=6, n_outer=8)


def _mapping(x, y):
    return (x + 0.04 * y ** 3 + 0.02 * x * y - 0.01 * x ** 3 * y,
            y + 0.03 * x * x * y - 0.01 * x * y ** 3 + 0.05 * x * x)


def _state(prm, seed):
    # random smooth perturbation of the free stream
    def f(x, y):
        q = fields.random_smooth_state(x, y, seed=seed, amp=0.05, scale=2.0, rho0=prm.rho_inf, p0=prm.p_inf,
                                       u0=prm.u_inf, v0=prm.v_inf, gamma=prm.gamma)
        return q
    return f


@pytest.mark.parametrize("N", [3, 4, 5, 6])
@pytest.mark.parametrize("viscous", [0, 1])
@pytest.mark.parametrize("precision", [0, 1])
def test_residual_cubic_channel_all_conditions(ssd, oracle_mod, N, viscous, precision):
    m = meshes.channel_mesh(5, 3, 3.0, 2.0, tags=(BC_INLET, BC_OUTLET, BC_SLIP, BC_SLIP), mapping=_mapping,
                            cubic=True)
    prm = FlowParams(gamma=1.4, Rgas=1.0, mu=0.02 * viscous, viscous=viscous, rho_inf=1.1, u_inf=0.6,
                     v_inf=-0.25, p_inf=0.9)
    s, o = ssd.Solver(m, N - 1, prm, precision=precision), oracle_mod.Oracle(m, N, prm)
    Q = o.state_from(_state(prm, 17 + N))
    s.sd_set_state(Q)
    _check(s.sd_residual(), (o if precision else o.extended()).residual(Q, 0.0), TOL32_RESIDUAL if precision else TOL64)


@pytest.mark.parametrize("N", [3, 5])
@pytest.mark.parametrize("t", [0.0, 0.37, 4.1])
@pytest.mark.parametrize("viscous", [0, 1])
def test_residual_fp64_small_ellipse(ssd, oracle_mod, N, t, viscous):
    m = _small_ellipse()
    prm = ellipse_params(omega=0.3)
    prm.viscous = viscous
    s, o = ssd.Solver(m, N - 1, prm), oracle_mod.Oracle(m, N, prm)
    Q = o.state_from(_state(prm, 5))
    s.sd_set_state(Q)
    s.sd_set_time(t)
    _check(s.sd_residual(), o.extended().residual(Q, t), TOL64)


@pytest.mark.parametrize("viscous", [0, 1])
def test_residual_fp32_small_ellipse(ssd, oracle_mod, viscous):
    m = _small_ellipse()
    prm = ellipse_params(omega=0.3)
    prm.viscous = viscous
    s, o = ssd.Solver(m, 4, prm, precision=1), oracle_mod.Oracle(m, 5, prm)
    Q = o.state_from(_state(prm, 6))
    s.sd_set_state(Q)
    s.sd_set_time(0.77)
    _check(s.sd_residual(), o.residual(Q, 0.77), TOL32_RESIDUAL)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("rk", [3, 5])
def test_steps_small_ellipse(ssd, oracle_mod, precision, rk):
    # impulsive start of the free stream past the rotating body
    m = _small_ellipse()
    prm = ellipse_params(omega=0.3)
    prm.rk_stages = rk
    s, o = ssd.Solver(m, 4, prm, precision=precision), oracle_mod.Oracle(m, 5, prm)
    Q = o.state_from(lambda x, y: fields.uniform(x, y, rho=1.0, u=1.0, v=0.0, p=prm.p_inf))
    dt, n = 2e-4, 10
    s.sd_set_state(Q)
    s.sd_step(dt, n)
    s.sd_sync()
    Qo, t = o.step(Q, 0.0, dt, n, rk_stages=rk)
    Qg = s.sd_get_state()
    if precision:
        # rho v starts at zero: it is the accumulated dt R of the first steps, so
        # its own relative L2 carries the FP32 residual tolerance; the state as a
        # whole, and every variable in max-norm, keep the FP32 state tolerance
        whole = np.sqrt(((Qg - Qo) ** 2).sum() / (Qo ** 2).sum())
        assert whole <= TOL32_STATE[0], whole
        assert (rel_err(Qg, Qo) <= TOL32_STATE[1]).all(), rel_err(Qg, Qo)
        _check(Qg, Qo, (TOL32_RESIDUAL[0], TOL32_STATE[1]))
    else:
        _check(Qg, Qo, TOL64)
    assert abs(s.sd_get_time() - t) < 1e-14


@pytest.mark.parametrize("precision", [0, 1])
def test_residual_full_ellipse_config(ssd, oracle_mod, precision):
    # the 20096-cell configuration at N = 5, whole residual against the oracle
    w = build_workload("ellipse_n5")
    s, o = ssd.Solver(w.mesh, w.N - 1, w.params, precision=precision), oracle_mod.Oracle(w.mesh, w.N, w.params)
    Q = o.state_from(_state(w.params, 9))
    s.sd_set_state(Q)
    s.sd_set_time(1.234)
    _check(s.sd_residual(), (o if precision else o.extended()).residual(Q, 1.234), TOL32_RESIDUAL if precision else TOL64)


def test_curved_mesh_errors(ssd):
    m = meshes.channel_mesh(3, 2, 3.0, 2.0, tags=(BC_INLET, BC_OUTLET, BC_SLIP, BC_SLIP), mapping=_mapping,
                            cubic=True)
    prm = FlowParams(rho_inf=1.0, u_inf=0.5, p_inf=1.0)
    bad = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in m.items()}
    bad["edge_nodes"][0, 1] = bad["edge_nodes"][0, 1][::-1].copy()
    with pytest.raises(ssd.SSDError, match="cubic edge nodes"):
        ssd.Solver(bad, 3, prm)
    bad = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in m.items()}
    bad["edge_arc"][0, 1] = 0
    with pytest.raises(ssd.SSDError, match="edge kinds differ"):
        ssd.Solver(bad, 3, prm)
    bad = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in m.items()}
    bad["bfaces"][0, 2] = 9
    with pytest.raises(ssd.SSDError, match="boundary tag"):
        ssd.Solver(bad, 3, prm)
    with pytest.raises(ssd.SSDError, match="free stream"):
        ssd.Solver(m, 3, FlowParams(rho_inf=0.0, p_inf=1.0))


@pytest.mark.parametrize("N", [3, 5])
@pytest.mark.parametrize("zone", [0, 1])
@pytest.mark.parametrize("precision", [0, 1])
def test_residual_adiabatic_box(ssd, oracle_mod, N, zone, precision):
    # closed box of adiabatic no-slip walls, stationary or rotating with the box
    m = meshes.channel_mesh(4, 3, 3.0, 2.0, tags=(BC_ADIABATIC,) * 4, mapping=_mapping, cubic=True, zone=zone)
    prm = FlowParams(gamma=1.4, Rgas=1.0, mu=0.05, viscous=1, T_wall=1.3, omega=0.8 * zone)
    s, o = ssd.Solver(m, N - 1, prm, precision=precision), oracle_mod.Oracle(m, N, prm)
    Q = o.state_from(lambda x, y: fields.random_smooth_state(x, y, seed=12, amp=0.2, scale=1.5))
    s.sd_set_state(Q)
    s.sd_set_time(0.3)
    _check(s.sd_residual(), (o if precision else o.extended()).residual(Q, 0.3), TOL32_RESIDUAL if precision else TOL64)


def _small_tank():
    return meshes.stirred_tank_mesh(n_theta_in=48, n_theta_out=40, layers_in=(3, 4, 3), layers_out=(3, 4))


def _tank_state(prm, seed):
    return lambda x, y: fields.random_smooth_state(x, y, seed=seed, amp=0.05, scale=2.0, p0=prm.Rgas, u0=0.1,
                                                   v0=-0.1, gamma=prm.gamma)


@pytest.mark.parametrize("N", [3, 4, 6])
@pytest.mark.parametrize("precision", [0, 1])
def test_residual_small_tank(ssd, oracle_mod, N, precision):
    m = _small_tank()
    prm = tank_params()
    s, o = ssd.Solver(m, N - 1, prm, precision=precision), oracle_mod.Oracle(m, N, prm)
    Q = o.state_from(_tank_state(prm, 21))
    s.sd_set_state(Q)
    s.sd_set_time(0.77)
    _check(s.sd_residual(), (o if precision else o.extended()).residual(Q, 0.77), TOL32_RESIDUAL if precision else TOL64)


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_steps_small_tank(ssd, oracle_mod, precision):
    # the tank starts at rest; the hub and blades set it moving
    m = _small_tank()
    prm = tank_params()
    s, o = ssd.Solver(m, 3, prm, precision=precision), oracle_mod.Oracle(m, 4, prm)
    Q = o.state_from(lambda x, y: fields.uniform(x, y, rho=1.0, p=prm.Rgas))
    dt, n = 5e-5, 10
    s.sd_set_state(Q)
    s.sd_step(dt, n)
    s.sd_sync()
    Qo, _ = o.step(Q, 0.0, dt, n)
    Qg = s.sd_get_state()
    if precision:
        # the momentum starts at zero (see test_steps_small_ellipse)
        whole = np.sqrt(((Qg - Qo) ** 2).sum() / (Qo ** 2).sum())
        assert whole <= TOL32_STATE[0], whole
        assert (rel_err(Qg, Qo) <= TOL32_STATE[1]).all(), rel_err(Qg, Qo)
    else:
        _check(Qg, Qo, TOL64)


@pytest.mark.parametrize("precision", [0, 1])
def test_residual_full_tank_config(ssd, oracle_mod, precision):
    w = build_workload("tank_n4")
    s, o = ssd.Solver(w.mesh, w.N - 1, w.params, precision=precision), oracle_mod.Oracle(w.mesh, w.N, w.params)
    Q = o.state_from(_tank_state(w.params, 22))
    s.sd_set_state(Q)
    s.sd_set_time(2.5)
    _check(s.sd_residual(), (o if precision else o.extended()).residual(Q, 2.5), TOL32_RESIDUAL if precision else TOL64)
