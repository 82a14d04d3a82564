"""Batched form: independent cases of different size, order and rotation rate
advanced together by one CUDA-graph launch per step must give exactly what
each case gives on its own, and agree with the oracle."""
import math

import numpy as np
import pytest

from helpers import small_rotor, small_twin
from ssd_inputs import fields, meshes
from ssd_inputs.workloads import FlowParams

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ssd():
    import paper_1503_02198_gb300 as pkg
    pkg.build()
    return pkg


def _cases():
    visc = FlowParams(gamma=1.4, Rgas=100.0 / 1.4, mu=0.1, prandtl=0.72, omega=1.0, viscous=1, T_wall=1.0)
    return [
        (small_rotor(), 2, FlowParams(omega=0.3)),
        (small_rotor(shift_R=0.05), 3, FlowParams(omega=0.9)),
        (meshes.couette_mesh(2, 12, 2, 16), 2, visc),
        (meshes.perturb_nodes(meshes.periodic_box_mesh(5, 2.0), 0.2, seed=1), 4, FlowParams()),
        (small_rotor(2), 5, FlowParams(omega=0.5)),
        (small_twin(omega2=-0.6, shift_L=0.05), 3, FlowParams(omega=0.7)),  # two rotating zones
    ]


def _state(solver, k, prm):
    if prm.viscous:
        return solver.state_from(lambda x, y: fields.uniform(x, y, rho=1.0, p=prm.Rgas))
    return solver.state_from(lambda x, y: fields.random_smooth_state(x, y, seed=10 + k, amp=0.1, scale=3.0))


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_equals_individual_runs(ssd, precision):
    cases = _cases()
    batch = ssd.Batch([c[0] for c in cases], [c[1] for c in cases], [c[2] for c in cases], precision=precision,
                      tune_dt=1e-4)
    dts = [1e-3, 7e-4, 2e-4, 1e-3, 5e-4, 8e-4]
    starts = []
    for k, (m, p, prm) in enumerate(cases):
        q = _state(batch.cases[k], k, prm)
        starts.append(q)
        batch.cases[k].sd_set_state(q)
    batch.sd_batch_step(dts, 5)
    batch.sd_batch_step(dts, 3)
    batch.sd_batch_sync()
    for k, (m, p, prm) in enumerate(cases):
        s = ssd.Solver(m, p, prm, precision=precision)
        s.sd_set_state(starts[k])
        s.sd_step(dts[k], 8)
        s.sd_sync()
        assert np.array_equal(batch.cases[k].sd_get_state(), s.sd_get_state()), k
        assert batch.cases[k].sd_get_time() == pytest.approx(8 * dts[k], rel=1e-14)
    batch.close()


def test_batch_case_matches_oracle(ssd, oracle_mod):
    cases = _cases()[:2]
    batch = ssd.Batch([c[0] for c in cases], [c[1] for c in cases], [c[2] for c in cases])
    m, p, prm = cases[1]
    o = oracle_mod.Oracle(m, p + 1, prm)
    q = o.state_from(lambda x, y: fields.isentropic_vortex(x, y, x0=1.0))
    batch.cases[0].sd_set_state(_state(batch.cases[0], 0, cases[0][2]))
    batch.cases[1].sd_set_state(q)
    batch.sd_batch_step([1e-3, 2e-3], 4)
    batch.sd_batch_sync()
    ref, _ = o.step(q, 0.0, 2e-3, 4)
    got = batch.cases[1].sd_get_state()
    l2 = np.sqrt(((got - ref) ** 2).sum(axis=(0, 2, 3)) / (ref ** 2).sum(axis=(0, 2, 3)))
    assert (l2 <= 1e-12).all(), l2
    batch.close()


def test_batch_reports_a_failing_case(ssd):
    cases = _cases()[:2]
    batch = ssd.Batch([c[0] for c in cases], [c[1] for c in cases], [c[2] for c in cases])
    q = _state(batch.cases[0], 0, cases[0][2])
    batch.cases[0].sd_set_state(q)
    bad = _state(batch.cases[1], 1, cases[1][2])
    bad[0, 0] = -1.0
    batch.cases[1].sd_set_state(bad)
    batch.sd_batch_step([1e-3, 1e-3], 1)
    with pytest.raises(ssd.SSDError) as ei:
        batch.sd_batch_sync()
    assert ei.value.code == ssd.SD_ERR_NONPHYSICAL
    batch.close()
