"""The FP32 form with the volume kernel's contractions on the tensor cores
(SD_PREC_FP32_TF32: interpolation to the flux points, Eq. Qt, and divergence,
Eqs. Ft / Gt, as 3xTF32 matrix multiplies) against the FP64 oracle, at the
FP32 form's tolerances: residuals on smooth and piecewise-constant states at
N = 3..6, and SSP-RK3 steps."""
import numpy as np
import pytest

from helpers import piecewise_constant, random_cell_states, rel_err, small_rotor, small_twin
from ssd_inputs import fields
from ssd_inputs.workloads import FlowParams

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
@pytest.mark.parametrize("which", ["smooth", "jumps"])
def test_residual_tf32(ssd, oracle_mod, N, which):
    m = small_rotor(shift_R=0.05)
    prm = FlowParams(omega=0.9)
    o = oracle_mod.Oracle(m, N, prm)
    if which == "smooth":
        Q = o.state_from(lambda x, y: fields.random_smooth_state(x, y, seed=N, amp=0.2, scale=3.0))
    else:
        Q = piecewise_constant(random_cell_states(o.E, seed=40 + N), N)
    s = ssd.Solver(m, N - 1, prm, precision=ssd.SD_PREC_FP32_TF32)
    s.sd_set_state(Q)
    s.sd_set_time(0.37)
    R = s.sd_residual()
    _check(R, o.residual(Q, 0.37), TOL32_RESIDUAL)
    # the same contractions on the FMA pipe agree to FP32 round-off
    f = ssd.Solver(m, N - 1, prm, precision=ssd.SD_PREC_FP32)
    f.sd_set_state(Q)
    f.sd_set_time(0.37)
    _check(R, f.sd_residual(), TOL32_RESIDUAL)
    s.close()
    f.close()


@pytest.mark.parametrize("N", [4, 6])
def test_steps_tf32(ssd, oracle_mod, N):
    m = small_twin()
    prm = FlowParams(omega=0.7)
    o = oracle_mod.Oracle(m, N, prm)
    Q = o.state_from(lambda x, y: fields.isentropic_vortex(x, y, x0=0.5))
    s = ssd.Solver(m, N - 1, prm, precision=ssd.SD_PREC_FP32_TF32)
    s.sd_set_state(Q)
    s.sd_step(1e-3, 10)
    s.sd_sync()
    q, _ = o.step(Q, 0.0, 1e-3, 10)
    _check(s.sd_get_state(), q, TOL32_STATE)
    s.close()


def test_tf32_not_offered_in_the_batch(ssd):
    m = small_rotor()
    with pytest.raises(ssd.SSDError) as ei:
        ssd.Batch([m], [2], [FlowParams(omega=0.5)], precision=ssd.SD_PREC_FP32_TF32)
    assert ei.value.code == ssd.SD_ERR_UNSUPPORTED
