"""Parity of the CUDA path with the oracle on states that jump across every
face: a random constant state per cell, so that each conforming face, each
periodic face and each mortar carries an O(1) jump and the dissipation term
of the Rusanov common flux (Sec. 3.1; on the mortars Sec. 3.2) enters every
common flux.  The oracle's Rusanov flux is pinned by tests/test_oracle_rusanov.py."""
import numpy as np
import pytest

from helpers import piecewise_constant, random_cell_states, rel_err, small_rotor, small_twin
from ssd_inputs import meshes
from ssd_inputs.workloads import FlowParams

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


def _mesh(which):
    if which == "rotor":
        return meshes.perturb_nodes(small_rotor(shift_R=0.05), 0.15, seed=5)
    return small_twin()


@pytest.mark.parametrize("which", ["rotor", "twin"])
@pytest.mark.parametrize("N", [3, 6])
@pytest.mark.parametrize("precision", [0, 1])
def test_residual_piecewise_constant(ssd, oracle_mod, which, N, precision):
    m = _mesh(which)
    prm = FlowParams(omega=0.9)
    o = oracle_mod.Oracle(m, N, prm)
    Q = piecewise_constant(random_cell_states(o.E, seed=31 + N), N)
    s = ssd.Solver(m, N - 1, prm, precision=precision)
    s.sd_set_state(Q)
    for t in (0.0, 0.77):
        s.sd_set_time(t)
        ref = (o.extended() if precision == 0 else o).residual(Q, t)
        _check(s.sd_residual(), ref, TOL64 if precision == 0 else TOL32_RESIDUAL)
    s.close()


@pytest.mark.parametrize("which", ["rotor", "twin"])
@pytest.mark.parametrize("precision", [0, 1])
def test_steps_from_piecewise_constant(ssd, oracle_mod, which, precision):
    N = 4
    m = _mesh(which)
    prm = FlowParams(omega=0.9)
    o = oracle_mod.Oracle(m, N, prm)
    Q = piecewise_constant(random_cell_states(o.E, seed=7), N)
    s = ssd.Solver(m, N - 1, prm, precision=precision)
    s.sd_set_state(Q)
    s.sd_set_time(0.3)
    dt = 2e-4
    s.sd_step(dt, 3)
    s.sd_sync()
    q, _ = o.step(Q, 0.3, dt, 3)
    _check(s.sd_get_state(), q, TOL64 if precision == 0 else TOL32_STATE)
    s.close()
