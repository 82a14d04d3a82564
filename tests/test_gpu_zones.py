"""Parity of the CUDA path with the FP64 oracle on meshes with several
rotating zones (each with its own centre, angular velocity and sliding
interface), through the C ABI.  Tolerances as in test_gpu_parity."""
import math

import numpy as np
import pytest

from helpers import rel_err, small_row, small_twin
from ssd_inputs import fields
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


def _state(o, seed):
    return o.state_from(lambda x, y: fields.random_smooth_state(x, y, seed=seed, amp=0.2, scale=2.0))


@pytest.mark.parametrize("N", [3, 4, 5, 6])
@pytest.mark.parametrize("t", [0.0, 0.37, 40.1])
def test_residual_fp64_two_zones(ssd, oracle_mod, N, t):
    m = small_twin(omega2=-0.6, shift_L=0.05, shift_R=-0.03)
    prm = FlowParams(omega=0.9)
    s, o = ssd.Solver(m, N - 1, prm), oracle_mod.Oracle(m, N, prm)
    Q = _state(o, N)
    s.sd_set_state(Q)
    s.sd_set_time(t)
    _check(s.sd_residual(), o.extended().residual(Q, t), TOL64)
    s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_residual_two_zones_viscous(ssd, oracle_mod, precision):
    m = small_twin(omega2=0.7, shift_L=0.02)
    prm = FlowParams(omega=-0.4, viscous=1, mu=0.03)
    s, o = ssd.Solver(m, 3, prm, precision=precision), oracle_mod.Oracle(m, 4, prm)
    Q = _state(o, 7)
    s.sd_set_state(Q)
    s.sd_set_time(0.61)
    _check(s.sd_residual(), (o.extended() if precision == 0 else o).residual(Q, 0.61), TOL64 if precision == 0 else TOL32_RESIDUAL)
    s.close()


@pytest.mark.parametrize("precision,N", [(1, 4), (1, 6), (2, 5)])
def test_residual_fp32_two_zones(ssd, oracle_mod, precision, N):
    m = small_twin(omega2=-0.6, shift_L=0.05)
    prm = FlowParams(omega=0.9)
    s, o = ssd.Solver(m, N - 1, prm, precision=precision), oracle_mod.Oracle(m, N, prm)
    Q = _state(o, 11)
    s.sd_set_state(Q)
    s.sd_set_time(0.37)
    _check(s.sd_residual(), o.residual(Q, 0.37), TOL32_RESIDUAL)
    s.close()


def test_four_zones_residual_and_steps(ssd, oracle_mod):
    # the most rotating zones a mesh may have, each with its own rate and face count
    m = small_row(4, (-0.6, 0.3, 1.1), shift_L=0.1, n_cores=(4, 3, 5, 2))
    prm = FlowParams(omega=0.9)
    s, o = ssd.Solver(m, 3, prm), oracle_mod.Oracle(m, 4, prm)
    Q = _state(o, 5)
    s.sd_set_state(Q)
    s.sd_set_time(2.3)
    _check(s.sd_residual(), o.extended().residual(Q, 2.3), TOL64)
    s.sd_step(2e-3, 3)
    s.sd_sync()
    q_ref, t_ref = o.step(Q, 2.3, 2e-3, 3)
    assert s.sd_get_time() == t_ref
    _check(s.sd_get_state(), q_ref, TOL64)
    s.close()


def test_five_zones_rejected(ssd):
    m = small_row(5, (-0.6, 0.3, 1.1, 0.2))
    with pytest.raises(ssd.SSDError) as ei:
        ssd.Solver(m, 2, FlowParams())
    assert ei.value.code == ssd.SD_ERR_ARG


def test_zone_mesh_errors_rejected(ssd):
    m = small_twin()
    bad = dict(m)
    az = m["elem_arc_zone"].copy()
    az[np.flatnonzero(m["elem_zone"] == 2)[0]] = 1
    bad["elem_arc_zone"] = az
    with pytest.raises(ssd.SSDError) as ei:
        ssd.Solver(bad, 2, FlowParams())
    assert ei.value.code == ssd.SD_ERR_MESH
    bad = dict(m)
    z2 = dict(m["zones"][0])
    z2["ifaces_L"] = m["ifaces_L"]
    bad["zones"] = [z2]
    with pytest.raises(ssd.SSDError):
        ssd.Solver(bad, 2, FlowParams())


@pytest.mark.parametrize("precision,N,rk", [(0, 4, 3), (0, 3, 5), (1, 6, 3), (2, 4, 3)])
def test_steps_two_zones(ssd, oracle_mod, precision, N, rk):
    m = small_twin(omega2=-math.pi / 4, shift_L=0.02)
    prm = FlowParams(omega=math.pi / 4, rk_stages=rk)
    s, o = ssd.Solver(m, N - 1, prm, precision=precision), oracle_mod.Oracle(m, N, prm)
    Q = o.state_from(lambda x, y: fields.isentropic_vortex(x, y, x0=0.5, y0=0.3))
    dt, n = (2e-3, 4) if precision == 0 else (1e-3, 10)
    s.sd_set_state(Q)
    s.sd_set_time(0.2)
    s.sd_step(dt, n)
    s.sd_sync()
    q_ref, t_ref = o.step(Q, 0.2, dt, n, rk_stages=rk)
    assert s.sd_get_time() == t_ref
    _check(s.sd_get_state(), q_ref, TOL64 if precision == 0 else TOL32_STATE)
    s.close()


def test_sp_coords_two_zones(ssd, oracle_mod):
    m = small_twin(omega2=-0.7)
    s, o = ssd.Solver(m, 3, FlowParams(omega=0.3)), oracle_mod.Oracle(m, 4, FlowParams(omega=0.3))
    for t in (0.0, 1.7):
        xy = s.sd_sp_coords(t)
        x, y = o.sp_coords(t)
        np.testing.assert_allclose(xy[..., 0], x, atol=1e-13)
        np.testing.assert_allclose(xy[..., 1], y, atol=1e-13)
    s.close()


def test_full_size_twin_rotor(ssd, oracle_mod):
    # the two-zone workload at full size (123,450 quads, N = 6): the FP64
    # residual at every point, and one captured-graph FP32 step against the
    # oracle's step from the same state
    w = build_workload("twin_rotor_n6")
    o = oracle_mod.Oracle(w.mesh, w.N, w.params)
    Q = o.state_from(lambda x, y: fields.random_smooth_state(x, y, seed=21, amp=0.2, scale=4.0))
    s = ssd.Solver(w.mesh, w.N - 1, w.params)
    s.sd_set_state(Q)
    s.sd_set_time(0.8)
    R = s.sd_residual()
    Rr = o.residual(Q, 0.8)
    _check(R, Rr, (1e-11, 1e-11))
    s.close()
    s = ssd.Solver(w.mesh, w.N - 1, w.params, precision=1)
    Qv = o.state_from(lambda x, y: fields.isentropic_vortex(x, y, x0=6.5, y0=0.5))
    s.sd_set_state(Qv)
    s.sd_step(w.cfl_dt, 1)
    s.sd_sync()
    q_ref, _ = o.step(Qv, 0.0, w.cfl_dt, 1)
    _check(s.sd_get_state(), q_ref, TOL32_STATE)
    s.close()
