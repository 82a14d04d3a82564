"""FP32 state storage (SD_PREC_FP32S) through the C ABI.

The residual arithmetic is the FP32 path's, which reads only the float part
of its double-float state, so for the same input both give bit-identical
residuals.  Steps differ: each Runge-Kutta stage result is rounded to float
once (unit round-off u = 2^-24), so after n steps of an s-stage scheme the
state differs from the oracle by at most about n s u relative on top of the
FP32 path's own error; for the step counts below (n s <= 60) that stays within
the FP32 state tolerance of 1e-5."""
import numpy as np
import pytest

from helpers import rel_err, small_rotor
from ssd_inputs import fields, meshes
from ssd_inputs.workloads import FlowParams, ellipse_params

pytestmark = pytest.mark.gpu

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


@pytest.mark.parametrize("N", [3, 4, 5, 6])
@pytest.mark.parametrize("viscous", [0, 1])
def test_residual_equals_fp32_path_and_oracle(ssd, oracle_mod, N, viscous):
    m = small_rotor(shift_R=0.05)
    prm = FlowParams(omega=0.9, viscous=viscous, mu=0.02 * viscous)
    o = oracle_mod.Oracle(m, N, prm)
    Q = o.state_from(lambda x, y: fields.random_smooth_state(x, y, seed=N, amp=0.2, scale=3.0))
    s32 = ssd.Solver(m, N - 1, prm, precision=ssd.SD_PREC_FP32)
    s32s = ssd.Solver(m, N - 1, prm, precision=ssd.SD_PREC_FP32S)
    for s in (s32, s32s):
        s.sd_set_state(Q)
        s.sd_set_time(0.41)
    r32, r32s = s32.sd_residual(), s32s.sd_residual()
    assert np.array_equal(r32, r32s)
    _check(r32s, o.residual(Q, 0.41), TOL32_RESIDUAL)


@pytest.mark.parametrize("N", [3, 6])
@pytest.mark.parametrize("rk", [3, 5])
def test_steps_rotor(ssd, oracle_mod, N, rk):
    m = small_rotor(shift_R=0.05)
    prm = FlowParams(omega=0.9, rk_stages=rk)
    o = oracle_mod.Oracle(m, N, prm)
    Q = o.state_from(lambda x, y: fields.isentropic_vortex(x, y, x0=1.0, y0=-0.5))
    s = ssd.Solver(m, N - 1, prm, precision=ssd.SD_PREC_FP32S)
    s.sd_set_state(Q)
    dt, n = 0.004, 12
    s.sd_step(dt, n)
    s.sd_sync()
    Qo, t = o.step(Q, 0.0, dt, n, rk_stages=rk)
    _check(s.sd_get_state(), Qo, TOL32_STATE)
    assert abs(s.sd_get_time() - t) < 1e-14


def test_state_is_float_rounded(ssd, oracle_mod):
    # set_state / get_state round to the nearest float (no low part is kept)
    m = small_rotor()
    prm = FlowParams(omega=0.5)
    o = oracle_mod.Oracle(m, 4, prm)
    Q = o.state_from(lambda x, y: fields.random_smooth_state(x, y, seed=2, amp=0.2, scale=3.0))
    s = ssd.Solver(m, 3, prm, precision=ssd.SD_PREC_FP32S)
    s.sd_set_state(Q)
    assert np.array_equal(s.sd_get_state(), Q.astype(np.float32).astype(np.float64))


def test_steps_couette_viscous(ssd, oracle_mod):
    m = meshes.couette_mesh(2, 12, 2, 16)
    U, c = 1.0, 10.0
    prm = FlowParams(gamma=1.4, Rgas=c * c / 1.4, mu=U / 10.0, omega=1.0, viscous=1, T_wall=1.0)
    o = oracle_mod.Oracle(m, 4, prm)
    Q = o.state_from(lambda x, y: fields.random_smooth_state(x, y, seed=4, amp=0.02, p0=prm.Rgas, u0=0.0,
                                                            v0=0.0))
    s = ssd.Solver(m, 3, prm, precision=ssd.SD_PREC_FP32S)
    s.sd_set_state(Q)
    dt, n = 2e-5, 15
    s.sd_step(dt, n)
    s.sd_sync()
    Qo, _ = o.step(Q, 0.0, dt, n)
    _check(s.sd_get_state(), Qo, TOL32_STATE)


def test_steps_small_ellipse(ssd, oracle_mod):
    m = meshes.ellipse_mesh(n_theta=32, n_inner=6, n_outer=8)
    prm = ellipse_params(omega=0.3)
    o = oracle_mod.Oracle(m, 5, prm)
    Q = o.state_from(lambda x, y: fields.ellipse_start(x, y, prm.rho_inf, prm.u_inf, prm.v_inf, prm.p_inf,
                                                       prm.omega))
    s = ssd.Solver(m, 4, prm, precision=ssd.SD_PREC_FP32S)
    s.sd_set_state(Q)
    dt, n = 2e-4, 10
    s.sd_step(dt, n)
    s.sd_sync()
    Qo, _ = o.step(Q, 0.0, dt, n)
    _check(s.sd_get_state(), Qo, TOL32_STATE)
