"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

FP64 path: residual and steps within 1e-12 relative L2 of the oracle per
conservative variable, and within 2e-11 of the largest magnitude of that
variable at every point (round-off of two independent FP64 evaluations,
amplified by the flux-derivative weights, reaches ~2e-12 of max|R| at N=5-6).
FP32 path: within the tolerances derived in the design notes.
"""
import math

import numpy as np
import pytest

from helpers import rel_err, small_rotor
from ssd_inputs import fields, meshes
from ssd_inputs.workloads import FlowParams, build_workload

pytestmark = pytest.mark.gpu

TOL64 = (1e-12, 1e-12)  # FP64 residuals against the extended-precision oracle; states against the FP64 oracle
# FP32 residual: the same amplification of round-off as in FP64 (~1e4 ulp of
# max|R| at N=5-6) applied to the FP32 unit round-off 6e-8
TOL32_RESIDUAL = (5e-5, 5e-4)
# FP32 state after steps (state and Runge-Kutta accumulation stay FP64)
TOL32_STATE = (1e-5, 1e-5)


@pytest.fixture(scope="module")
def ssd():
    import paper_1503_02198_gb300 as pkg
    pkg.build()
    return pkg


def _pair(ssd, oracle_mod, mesh, N, prm, precision=0):
    return ssd.Solver(mesh, N - 1, prm, precision=precision), oracle_mod.Oracle(mesh, N, prm)


def _check(a, b, tol):
    l2 = np.sqrt(((a - b) ** 2).sum(axis=(0, 2, 3)) / (b ** 2).sum(axis=(0, 2, 3)))
    mx = rel_err(a, b)
    assert (l2 <= tol[0]).all() and (mx <= tol[1]).all(), (l2, mx)


@pytest.mark.parametrize("N", [3, 4, 5, 6])
@pytest.mark.parametrize("t", [0.0, 0.37, 5.123])
def test_residual_fp64_rotor(ssd, oracle_mod, N, t):
    m = small_rotor(shift_R=0.05)
    prm = FlowParams(omega=0.9)
    s, o = _pair(ssd, oracle_mod, m, N, prm)
    Q = o.state_from(lambda x, y: fields.random_smooth_state(x, y, seed=N, amp=0.2, scale=3.0))
    s.sd_set_state(Q)
    s.sd_set_time(t)
    _check(s.sd_residual(), o.extended().residual(Q, t), TOL64)


@pytest.mark.parametrize("N", [3, 5])
def test_residual_fp64_aligned_and_degenerate_mortars(ssd, oracle_mod, N):
    # equal face counts, nodes coincide at theta = k * 2 pi / 24: zero-length mortars
    m = small_rotor(n_hole=6, n_core=6)
    prm = FlowParams(omega=1.0)
    s, o = _pair(ssd, oracle_mod, m, N, prm)
    Q = o.state_from(lambda x, y: fields.isentropic_vortex(x, y, x0=1.0, y0=-2.0))
    s.sd_set_state(Q)
    for t in (0.0, 2 * math.pi / 24, 3 * 2 * math.pi / 24 + 1e-9):
        s.sd_set_time(t)
        _check(s.sd_residual(), o.extended().residual(Q, t), TOL64)


def test_residual_fp64_periodic_box_no_interface(ssd, oracle_mod):
    m = meshes.perturb_nodes(meshes.periodic_box_mesh(6, 2.0), 0.2, seed=9)
    s, o = _pair(ssd, oracle_mod, m, 4, FlowParams())
    Q = o.state_from(lambda x, y: fields.random_smooth_state(x, y, seed=3, amp=0.3))
    s.sd_set_state(Q)
    _check(s.sd_residual(), o.extended().residual(Q, 0.0), TOL64)


def test_residual_fp64_walls_inviscid(ssd, oracle_mod):
    # Couette annulus with Euler fluxes: rotating and stationary walls, curved cells
    m = meshes.couette_mesh(2, 12, 2, 16)
    prm = FlowParams(omega=0.5, Rgas=2.0, T_wall=1.3)
    s, o = _pair(ssd, oracle_mod, m, 3, prm)
    Q = o.state_from(lambda x, y: fields.random_smooth_state(x, y, seed=4, amp=0.1, u0=0.1, v0=0.2,
                                                             p0=2.5))
    s.sd_set_state(Q)
    s.sd_set_time(0.77)
    _check(s.sd_residual(), o.extended().residual(Q, 0.77), TOL64)


def test_sp_coords_match_oracle(ssd, oracle_mod):
    m = small_rotor()
    s, o = _pair(ssd, oracle_mod, m, 4, FlowParams(omega=0.3))
    for t in (0.0, 1.7):
        xy = s.sd_sp_coords(t)
        x, y = o.sp_coords(t)
        np.testing.assert_allclose(xy[..., 0], x, atol=1e-13)
        np.testing.assert_allclose(xy[..., 1], y, atol=1e-13)


@pytest.mark.parametrize("N", [3, 6])
def test_steps_fp64(ssd, oracle_mod, N):
    m = small_rotor(shift_L=0.02)
    prm = FlowParams(omega=math.pi / 4)
    s, o = _pair(ssd, oracle_mod, m, N, prm)
    Q = o.state_from(lambda x, y: fields.isentropic_vortex(x, y, x0=2.0))
    dt = 2e-3
    s.sd_set_state(Q)
    s.sd_set_time(0.1)
    s.sd_step(dt, 4)
    s.sd_sync()
    q_ref, t_ref = o.step(Q, 0.1, dt, 4)
    assert s.sd_get_time() == t_ref
    _check(s.sd_get_state(), q_ref, TOL64)
    # resuming from the returned state and time continues identically (checkpoint)
    q_mid = s.sd_get_state()
    s.sd_step(dt, 2)
    s.sd_sync()
    a = s.sd_get_state()
    s2 = ssd.Solver(m, N - 1, prm)
    s2.sd_set_state(q_mid)
    s2.sd_set_time(t_ref)
    s2.sd_step(dt, 2)
    s2.sd_sync()
    assert np.array_equal(a, s2.sd_get_state())


@pytest.mark.parametrize("N", [3, 4, 6])
def test_residual_fp32_rotor(ssd, oracle_mod, N):
    m = small_rotor(shift_R=0.05)
    prm = FlowParams(omega=0.9)
    s, o = _pair(ssd, oracle_mod, m, N, prm, precision=1)
    Q = o.state_from(lambda x, y: fields.isentropic_vortex(x, y, x0=1.0))
    s.sd_set_state(Q)
    s.sd_set_time(0.37)
    _check(s.sd_residual(), o.residual(Q, 0.37), TOL32_RESIDUAL)


@pytest.mark.parametrize("N", [3, 6])
def test_steps_fp32(ssd, oracle_mod, N):
    m = small_rotor(shift_L=0.02)
    prm = FlowParams(omega=math.pi / 4)
    s, o = _pair(ssd, oracle_mod, m, N, prm, precision=1)
    Q = o.state_from(lambda x, y: fields.isentropic_vortex(x, y, x0=2.0))
    dt = 1e-3
    s.sd_set_state(Q)
    s.sd_step(dt, 20)
    s.sd_sync()
    q_ref, _ = o.step(Q, 0.0, dt, 20)
    _check(s.sd_get_state(), q_ref, TOL32_STATE)


def test_full_size_vortex_residual_fp64(ssd, oracle_mod):
    w = build_workload("vortex_n4")
    s, o = _pair(ssd, oracle_mod, w.mesh, w.N, w.params)
    Q = o.state_from(lambda x, y: fields.isentropic_vortex(x, y))
    s.sd_set_state(Q)
    s.sd_set_time(1.1)
    _check(s.sd_residual(), o.extended().residual(Q, 1.1), TOL64)


@pytest.mark.parametrize("precision", [0, 1])
def test_negative_pressure_is_reported(ssd, precision):
    # positive density, kinetic energy above the total energy in one element:
    # p = (gamma - 1) (E - |m|^2 / (2 rho)) < 0
    m = small_rotor()
    s = ssd.Solver(m, 2, FlowParams(omega=0.5), precision=precision)
    Q = s.state_from(lambda x, y: fields.uniform(x, y))
    Q[5, 1] = 3.0 * Q[5, 0]  # momentum 3 rho per unit density
    Q[5, 3] = 0.5 * Q[5, 0]  # E = rho / 2 < |m|^2 / (2 rho) = 4.5 rho
    s.sd_set_state(Q)
    s.sd_step(1e-4, 1)
    with pytest.raises(ssd.SSDError) as ei:
        s.sd_sync()
    assert ei.value.code == ssd.SD_ERR_NONPHYSICAL
    s.sd_set_state(s.state_from(lambda x, y: fields.uniform(x, y)))
    s.sd_step(1e-4, 1)
    s.sd_sync()


def test_non_physical_state_is_reported(ssd, oracle_mod):
    m = small_rotor()
    s = ssd.Solver(m, 2, FlowParams(omega=0.5))
    Q = s.state_from(lambda x, y: fields.uniform(x, y))
    Q[3, 0] = -1.0  # negative density in one element
    s.sd_set_state(Q)
    s.sd_step(1e-3, 1)
    with pytest.raises(ssd.SSDError) as ei:
        s.sd_sync()
    assert ei.value.code == ssd.SD_ERR_NONPHYSICAL
    # the flag is cleared once reported; a good state steps cleanly again
    s.sd_set_state(s.state_from(lambda x, y: fields.uniform(x, y)))
    s.sd_step(1e-3, 1)
    s.sd_sync()


def test_bad_mesh_rejected_by_library(ssd):
    m = dict(small_rotor())
    m["pfaces"] = m["pfaces"][1:]
    with pytest.raises(ssd.SSDError) as ei:
        ssd.Solver(m, 2, FlowParams())
    assert ei.value.code == ssd.SD_ERR_MESH
    m = dict(small_rotor())
    en = m["elem_nodes"].copy()
    en[0] = en[0][::-1]  # clockwise cell
    m["elem_nodes"] = en
    with pytest.raises(ssd.SSDError):
        ssd.Solver(m, 2, FlowParams())


@pytest.fixture(scope="module")
def rotor_full(oracle_mod):
    w = build_workload("rotor_n6")
    o = oracle_mod.Oracle(w.mesh, w.N, w.params)
    Q = o.state_from(lambda x, y: fields.isentropic_vortex(x, y, x0=3.0, y0=1.0))
    return w, o, Q


def test_full_size_rotor_residual_fp64(ssd, rotor_full):
    # the bench workload at full size (246,900 quads, N = 6); a state whose
    # residual is O(1) everywhere (with the vortex most of the domain is free
    # stream, where the true residual is below round-off and no relative
    # measure is meaningful)
    # At h = 0.08 and N = 6 each SP residual is a weighted difference of flux
    # values up to ~1e3 times larger than itself, so two independent FP64
    # evaluations differ by ~3e-12 relative L2 (the round-off floor).  Where
    # the divergence terms do not cancel among themselves (straight cells of
    # the stationary zone) the arithmetic bounds the difference per point:
    # |dR| <= c u S with S = sum of the magnitudes of the divergence terms (from
    # the oracle), u = 2^-53, c = 128 (2(N+1) terms, each flux value carrying a
    # few tens of u, two independent evaluations).
    w, o, _ = rotor_full
    Q = o.state_from(lambda x, y: fields.random_smooth_state(x, y, seed=21, amp=0.2, scale=4.0))
    s = ssd.Solver(w.mesh, w.N - 1, w.params)
    s.sd_set_state(Q)
    s.sd_set_time(0.8)
    R = s.sd_residual()
    Rr, S = o.residual_with_scale(Q, 0.8)
    m = w.mesh
    plain = (m["edge_arc"].sum(axis=1) == 0) & (m["elem_zone"] == 0)
    ratio = np.abs(R - Rr)[plain] / (2.0 ** -53 * S[plain])
    assert ratio.max() <= 128.0, ratio.max()
    _check(R, Rr, (1e-11, 1e-11))
    s.close()


def test_full_size_rotor_step_fp32(ssd, rotor_full):
    # one captured-graph SSP-RK3 step of the FP32 path, as the benchmark times it
    w, o, Q = rotor_full
    s = ssd.Solver(w.mesh, w.N - 1, w.params, precision=1)
    s.sd_set_state(Q)
    s.sd_step(w.cfl_dt, 1)
    s.sd_sync()
    q_ref, _ = o.step(Q, 0.0, w.cfl_dt, 1)
    _check(s.sd_get_state(), q_ref, TOL32_STATE)
    s.close()


@pytest.mark.parametrize("precision,N", [(0, 3), (0, 5), (1, 4)])
def test_steps_rk54(ssd, oracle_mod, precision, N):
    # the five-stage fourth-order SSP Runge-Kutta of Sec. 4
    m = small_rotor(shift_L=0.02)
    prm = FlowParams(omega=math.pi / 4, rk_stages=5)
    s, o = _pair(ssd, oracle_mod, m, N, prm, precision=precision)
    Q = o.state_from(lambda x, y: fields.isentropic_vortex(x, y, x0=2.0))
    dt = 2e-3
    s.sd_set_state(Q)
    s.sd_set_time(0.05)
    s.sd_step(dt, 4)
    s.sd_sync()
    q_ref, t_ref = o.step(Q, 0.05, dt, 4, rk_stages=5)
    assert abs(s.sd_get_time() - t_ref) < 1e-15
    _check(s.sd_get_state(), q_ref, TOL64 if precision == 0 else TOL32_STATE)


@pytest.mark.parametrize("omega,t", [(0.9, 100.0), (-0.7, 123.4), (0.0, 3.0)])
def test_residual_fp64_many_turns_clockwise_and_still(ssd, oracle_mod, omega, t):
    # rotation angles of many turns (theta = 90 rad), clockwise rotation
    # (theta = -86 rad) and a sliding interface that does not move
    m = small_rotor(shift_R=0.05)
    prm = FlowParams(omega=omega)
    s, o = _pair(ssd, oracle_mod, m, 4, prm)
    Q = o.state_from(lambda x, y: fields.random_smooth_state(x, y, seed=31, amp=0.2, scale=3.0))
    s.sd_set_state(Q)
    s.sd_set_time(t)
    _check(s.sd_residual(), o.extended().residual(Q, t), TOL64)


@pytest.mark.parametrize("precision", [0, 1])
def test_steps_clockwise_from_late_time(ssd, oracle_mod, precision):
    m = small_rotor(shift_L=0.03)
    prm = FlowParams(omega=-0.8)
    s, o = _pair(ssd, oracle_mod, m, 5, prm, precision=precision)
    Q = o.state_from(lambda x, y: fields.isentropic_vortex(x, y, x0=-1.0, y0=0.5))
    t0, dt, n = 50.0, 0.004, 10
    s.sd_set_state(Q)
    s.sd_set_time(t0)
    s.sd_step(dt, n)
    s.sd_sync()
    Qo, t = o.step(Q, t0, dt, n)
    _check(s.sd_get_state(), Qo, TOL32_STATE if precision else TOL64)
    assert abs(s.sd_get_time() - t) < 1e-12


def test_zero_steps_change_nothing(ssd, oracle_mod):
    m = small_rotor()
    s, o = _pair(ssd, oracle_mod, m, 3, FlowParams(omega=0.5))
    Q = o.state_from(lambda x, y: fields.random_smooth_state(x, y, seed=4, amp=0.1, scale=3.0))
    s.sd_set_state(Q)
    s.sd_set_time(1.5)
    s.sd_step(0.01, 0)
    s.sd_sync()
    assert np.array_equal(s.sd_get_state(), Q) and s.sd_get_time() == 1.5


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_pinned_and_pageable_host_buffers_agree(ssd, oracle_mod, precision):
    # a pinned host buffer is read / written by the conversion kernels directly,
    # a pageable one goes through a staged copy: both must give the same bits
    import torch
    m = small_rotor(shift_R=0.05)
    prm = FlowParams(omega=0.9)
    o = oracle_mod.Oracle(m, 4, prm)
    Q = o.state_from(lambda x, y: fields.random_smooth_state(x, y, seed=8, amp=0.2, scale=3.0))
    a = ssd.Solver(m, 3, prm, precision=precision)
    b = ssd.Solver(m, 3, prm, precision=precision)
    a.sd_set_state(Q)                                   # numpy: pageable
    pin = torch.from_numpy(Q.copy()).pin_memory()
    b.sd_set_state(pin)                                 # pinned
    for s in (a, b):
        s.sd_step(1e-3, 2)
        s.sd_sync()
    qa = a.sd_get_state()
    out = torch.empty(Q.shape, dtype=torch.float64).pin_memory()
    b.sd_get_state(out)
    assert np.array_equal(qa, out.numpy())
    a.close()
    b.close()


@pytest.mark.parametrize("precision,viscous", [(0, 0), (1, 0), (1, 1)])
def test_profiled_steps_equal_graph_steps(ssd, oracle_mod, precision, viscous):
    # sd_profile_step runs the mortar flux as its own launch (to time it);
    # sd_step runs it inside the face launch of the same pass: the same
    # arithmetic, so the same bits
    m = small_rotor(shift_R=0.05)
    prm = FlowParams(omega=0.9, viscous=viscous, mu=0.02 * viscous)
    o = oracle_mod.Oracle(m, 4, prm)
    Q = o.state_from(lambda x, y: fields.random_smooth_state(x, y, seed=12, amp=0.2, scale=3.0))
    a = ssd.Solver(m, 3, prm, precision=precision)
    b = ssd.Solver(m, 3, prm, precision=precision)
    for s in (a, b):
        s.sd_set_state(Q)
        s.sd_set_time(0.3)
    a.sd_step(1e-3, 3)
    a.sd_sync()
    b.sd_profile_step(1e-3, reps=3)
    assert a.sd_get_time() == b.sd_get_time()
    assert np.array_equal(a.sd_get_state(), b.sd_get_state())
    a.close()
    b.close()
