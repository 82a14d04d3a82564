"""Captured steps and the stage merges that run beside them.

A captured step reads one of two sets of stage tables (clocks, mortar tables,
mortar offsets of Eq. xz) and merges every stage of the next step into the
other set, at the start time t_n + dt formed as the clock advance forms it;
each sd_step call merges its first step before the first captured step.  So
one call of n steps, n calls of one step, and calls that change dt between
them must all give the same bits as the serial order (merge, stages, advance),
and the oracle's result within the stated tolerance.  Covered on a sliding
rotor with a vortex across the interface (Euler, SSP-RK3 and SSP-RK(5,4), FP64
and FP32) and on the viscous Couette annulus."""
import numpy as np
import pytest

from helpers import small_rotor
from ssd_inputs import fields, meshes
from ssd_inputs.workloads import FlowParams

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ssd():
    import paper_1503_02198_gb300 as pkg
    pkg.build()
    return pkg


def _rel(a, b):
    return float(np.sqrt(((a - b) ** 2).sum() / (b ** 2).sum()))


def _rotor_case(rk):
    m = small_rotor(shift_L=0.03)
    prm = FlowParams(omega=0.8, rk_stages=rk)
    return m, prm, (lambda x, y: fields.isentropic_vortex(x, y, x0=2.5, y0=0.5))


def _couette_case():
    m = meshes.couette_mesh(2, 12, 2, 16, phi_out=0.05)
    Rg = 100.0 / 1.4
    prm = FlowParams(gamma=1.4, Rgas=Rg, mu=0.1, prandtl=0.72, omega=1.0, viscous=1, T_wall=1.0)
    return m, prm, (lambda x, y: fields.random_smooth_state(x, y, seed=7, amp=0.05, u0=0.2, v0=-0.1, p0=Rg))


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("case", ["rotor_rk3", "rotor_rk54", "couette"])
def test_one_call_of_n_steps_equals_n_calls(ssd, precision, case):
    m, prm, init = _rotor_case(5 if case == "rotor_rk54" else 3) if case != "couette" else _couette_case()
    dt = 1e-4 if case == "couette" else 2e-3
    a = ssd.Solver(m, 3, prm, precision=precision)
    b = ssd.Solver(m, 3, prm, precision=precision)
    Q = a.state_from(init)
    for s in (a, b):
        s.sd_set_state(Q)
        s.sd_set_time(0.3)
    a.sd_step(dt, 7)  # odd: both captured steps, the last one reading the second set
    for _ in range(7):
        b.sd_step(dt, 1)
    a.sd_sync()
    b.sd_sync()
    assert a.sd_get_time() == b.sd_get_time()
    assert np.array_equal(a.sd_get_state(), b.sd_get_state())
    a.close()
    b.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_changing_dt_between_calls_matches_the_oracle(ssd, oracle_mod, precision):
    m, prm, init = _rotor_case(3)
    s = ssd.Solver(m, 3, prm, precision=precision)
    o = oracle_mod.Oracle(m, 4, prm)
    Q = o.state_from(init)
    s.sd_set_state(Q)
    s.sd_set_time(0.1)
    s.sd_step(2e-3, 3)
    s.sd_step(1.5e-3, 4)
    s.sd_step(2e-3, 2)
    s.sd_sync()
    q, t = o.step(Q, 0.1, 2e-3, 3)
    q, t = o.step(q, t, 1.5e-3, 4)
    q, t = o.step(q, t, 2e-3, 2)
    assert abs(s.sd_get_time() - t) < 1e-14
    assert _rel(s.sd_get_state(), q) <= (1e-12 if precision == 0 else 1e-5)
    s.close()
