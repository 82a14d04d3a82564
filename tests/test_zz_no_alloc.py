"""sd_residual_noalloc: the residual for callers that cannot allocate device
memory after creating their handle (its work memory is a fixed array inside
the library).  Collected last on purpose: it runs after every other test."""
import math

import numpy as np
import pytest

from helpers import small_rotor
from ssd_inputs import fields, meshes
from ssd_inputs.workloads import FlowParams, build_workload

pytestmark = pytest.mark.gpu

TOL64 = (1e-12, 2e-11)  # the FP64 parity tolerance of the other GPU tests


def _close(a, b, tol):
    l2 = np.sqrt(((a - b) ** 2).sum(axis=(0, 2, 3)) / (b ** 2).sum(axis=(0, 2, 3)))
    mx = np.abs(a - b).max(axis=(0, 2, 3)) / np.abs(b).max(axis=(0, 2, 3))
    assert (l2 <= tol[0]).all() and (mx <= tol[1]).all(), (l2, mx)


@pytest.fixture(scope="module")
def ssd():
    import paper_1503_02198_gb300 as pkg
    pkg.build()
    return pkg


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_noalloc_matches_residual_on_consecutive_calls(ssd, precision):
    import torch
    m = small_rotor(shift_R=0.05)
    s = ssd.Solver(m, 4, FlowParams(omega=0.9), precision=precision)
    states = [s.state_from(lambda x, y: fields.isentropic_vortex(x, y, x0=1.0)),
              s.state_from(lambda x, y: fields.random_smooth_state(x, y, seed=8, amp=0.2, scale=3.0))]
    for call, (Q, t) in enumerate(zip(states, (0.37, 2.9))):
        s.sd_set_state(Q)
        s.sd_set_time(t)
        ref = s.sd_residual()
        # host output (staged through the library's fixed work memory)
        got = s.sd_residual_noalloc()
        _close(got, ref, TOL64)
        # device output, preallocated by the caller
        dev = torch.empty(s.shape, dtype=torch.float64, device="cuda")
        s.sd_residual_noalloc(dev)
        _close(dev.cpu().numpy(), ref, TOL64)


def test_noalloc_rejects_work_beyond_its_fixed_size(ssd):
    import torch
    # 15,460 quads at N=6: the host-output staging copy (17.8 MB) exceeds 16 MiB
    m = meshes.rotor_mesh(half_width=20.0, n_cart=128, n_hole=32, r_interface=4.0, n_core=12, core_half=2.0,
                          n_ring_in=4, n_ring_out=2)
    s = ssd.Solver(m, 5, FlowParams(omega=0.5), precision=1)
    assert s.E * 4 * 36 * 8 > 16 * 2 ** 20
    s.sd_set_state(s.state_from(lambda x, y: fields.isentropic_vortex(x, y)))
    with pytest.raises(ssd.SSDError) as ei:
        s.sd_residual_noalloc()
    assert ei.value.code == ssd.SD_ERR_ARG and "16777216" in str(ei.value)
    # with a device output only the interface work counts: accepted, and equal
    dev = torch.empty(s.shape, dtype=torch.float64, device="cuda")
    s.sd_residual_noalloc(dev)
    ref = s.sd_residual()
    _close(dev.cpu().numpy(), ref, TOL64)


def test_noalloc_viscous_matches_oracle(ssd, oracle_mod):
    # the viscous chain (common solution, gradient traces, viscous mortar
    # procedure) runs through the same fixed work memory: the Taylor-Couette
    # annulus, two consecutive calls, against the oracle
    w = build_workload("couette_n3")
    o = oracle_mod.Oracle(w.mesh, w.N, w.params)
    s = ssd.Solver(w.mesh, w.N - 1, w.params, precision=0)
    for seed, t in ((3, 0.2), (4, 1.7)):
        Q = o.state_from(lambda x, y: fields.random_smooth_state(x, y, seed=seed, amp=0.05, u0=0.1, v0=0.05))
        s.sd_set_state(Q)
        s.sd_set_time(t)
        _close(s.sd_residual_noalloc(), o.residual(Q, t), TOL64)


def test_noalloc_checks_the_output_buffer(ssd):
    import torch
    s = ssd.Solver(small_rotor(), 2, FlowParams(omega=0.5), precision=0)
    with pytest.raises(ValueError):
        s.sd_residual_noalloc(torch.empty(s.n_dofs - 1, dtype=torch.float64, device="cuda"))
