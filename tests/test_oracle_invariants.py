"""Pins of the oracle's residual and time stepping against what the paper and
the mathematics fix: free-stream preservation, discrete conservation through
the moving mortar, exactness on linear fields with the ALE grid-velocity
terms, aligned mortars reducing to conforming faces, truncation-error
convergence on the exact vortex and Taylor-Couette solutions (Secs. 4.1,
4.2), and the third-order accuracy of the SSP Runge-Kutta step."""
import math

import numpy as np
import pytest

from helpers import face_kinds, neighbours_of, small_rotor, sp_weights
from ssd_inputs import fields, meshes
from ssd_inputs.workloads import FlowParams


def test_face_table_is_consistent(oracle_mod):
    m = small_rotor()
    o = oracle_mod.Oracle(m, 3, FlowParams(omega=0.7))
    kind, nbr, rev = o.face_info()
    assert (kind >= 0).all()
    conf = np.where((kind == 0) | (kind == 1))[0]
    assert (nbr[nbr[conf]] == conf).all()
    assert (kind == 3).sum() == len(m["ifaces_L"]) and (kind == 4).sum() == len(m["ifaces_R"])


def test_bad_mesh_is_rejected(oracle_mod):
    m = small_rotor()
    m = dict(m)
    m["pfaces"] = m["pfaces"][1:]  # a face with neither neighbour nor boundary condition
    with pytest.raises(ValueError):
        oracle_mod.Oracle(m, 3, FlowParams())


@pytest.mark.parametrize("N", [3, 4, 5])
@pytest.mark.parametrize("t", [0.0, 0.37, 2.9])
def test_free_stream_on_straight_cells(oracle_mod, N, t):
    # A uniform state is an exact steady solution; on straight-sided cells of the
    # rotating and stationary zones the SD residual must vanish to round-off,
    # including the grid-velocity terms (their divergence cancels exactly).
    m = meshes.perturb_nodes(small_rotor(), 0.15, seed=3)
    o = oracle_mod.Oracle(m, N, FlowParams(omega=math.pi / 4))
    Q = o.state_from(lambda x, y: fields.uniform(x, y, rho=1.2, u=0.3, v=-0.1, p=0.9))
    R = o.residual(Q, t)
    straight = m["edge_arc"].sum(axis=1) == 0
    assert np.abs(R[straight]).max() < 2e-12


@pytest.mark.parametrize("N", [3, 4])
def test_free_stream_error_on_curved_cells_converges(oracle_mod, N):
    errs = []
    for s in (1, 2, 4):
        m = small_rotor(s)
        o = oracle_mod.Oracle(m, N, FlowParams(omega=math.pi / 4))
        Q = o.state_from(lambda x, y: fields.uniform(x, y, rho=1.0, u=0.3, v=-0.1, p=1.0))
        errs.append(np.abs(o.residual(Q, 0.37)).max())
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert (rates > N - 1 - 0.3).all(), (errs, rates)


@pytest.mark.parametrize("N", [3, 4, 6])
@pytest.mark.parametrize("t", [0.0, 0.21, 1.3])
def test_discrete_conservation_through_sliding_interface(oracle_mod, N, t):
    # Periodic domain: sum_e sum_ij w_i w_j |J| dQ/dt = 0 for every variable
    # (conforming Rusanov fluxes cancel pointwise; Eq. prjF2 preserves the
    # integral of the mortar flux on both sides).
    m = small_rotor(shift_L=0.1234)
    o = oracle_mod.Oracle(m, N, FlowParams(omega=0.9))
    Q = o.state_from(lambda x, y: fields.random_smooth_state(x, y, seed=11, amp=0.2, scale=3.0))
    R = o.residual(Q, t)
    J = o.sp_jacobian()
    w = sp_weights(oracle_mod, N)
    total = np.einsum("evji,eji,j,i->v", R, J, w, w)
    scale = np.einsum("evji,eji,j,i->v", np.abs(R), J, w, w)
    assert (np.abs(total) < 1e-13 * scale).all(), total / scale


def test_discrete_conservation_viscous(oracle_mod):
    m = small_rotor()
    prm = FlowParams(omega=0.6, viscous=1, mu=0.05, Rgas=1.0, prandtl=0.72)
    o = oracle_mod.Oracle(m, 4, prm)
    Q = o.state_from(lambda x, y: fields.random_smooth_state(x, y, seed=5, amp=0.2, scale=3.0))
    R = o.residual(Q, 0.43)
    J = o.sp_jacobian()
    w = sp_weights(oracle_mod, 4)
    total = np.einsum("evji,eji,j,i->v", R, J, w, w)
    scale = np.einsum("evji,eji,j,i->v", np.abs(R), J, w, w)
    assert (np.abs(total) < 1e-13 * scale).all(), total / scale


@pytest.mark.parametrize("N", [3, 4])
def test_linear_field_exact_with_grid_velocity(oracle_mod, N):
    # rho linear in x, uniform velocity and pressure: every flux is bilinear in
    # x, y, reproduced exactly by the SD polynomials on straight cells, so
    # dQ/dt = -(U - u_g) dQ/dx with u_g = -omega (y - y_c) on the rotating zone.
    omega, t, U, V, b = 0.7, 0.31, 0.4, -0.2, 0.05
    m = meshes.perturb_nodes(small_rotor(2), 0.1, seed=5)
    o = oracle_mod.Oracle(m, N, FlowParams(omega=omega))
    x, y = o.sp_coords(t)
    Q = np.moveaxis(fields.conservative(1.0 + b * x, U, V, np.full_like(x, 1.0)), -1, 1).copy()
    R = o.residual(Q, t)
    dQdx = np.moveaxis(fields.conservative(np.full_like(x, b), U, V, np.zeros_like(x)), -1, 1)
    dQdx[:, 3] = 0.5 * b * (U * U + V * V)
    ug = np.where(m["elem_zone"][:, None, None] == 1, -omega * y, 0.0)
    expect = -(U - ug)[:, None] * dQdx
    special = face_kinds(m)
    ok = ~neighbours_of(m, special)
    assert ok.sum() > 50 and (m["elem_zone"][ok] == 1).sum() > 10
    np.testing.assert_allclose(R[ok], expect[ok], atol=2e-13)


def test_aligned_mortar_equals_conforming_face(oracle_mod):
    # With equal face counts on both sides and no rotation, every mortar is a
    # whole face (o = 0, s = 1): the mortar path must equal the conforming path.
    m = small_rotor(n_hole=6, n_core=6)
    assert len(m["ifaces_L"]) == len(m["ifaces_R"])
    # conforming copy: merge the interface nodes, one zone, no interface
    xy = m["xy"]
    en = m["elem_nodes"].copy()
    Lnodes = set()
    for e, f in m["ifaces_L"]:
        a, b = meshes.FACE_CORNERS[f]
        Lnodes.update([en[e, a], en[e, b]])
    Rnodes = set()
    for e, f in m["ifaces_R"]:
        a, b = meshes.FACE_CORNERS[f]
        Rnodes.update([en[e, a], en[e, b]])
    remap = {}
    for n in Lnodes:
        d = [(np.hypot(*(xy[n] - xy[r])), r) for r in Rnodes]
        dist, r = min(d)
        assert dist < 1e-12
        remap[n] = r
    en2 = np.vectorize(lambda n: remap.get(n, n))(en).astype(np.int32)
    m2 = dict(m)
    m2.update(elem_nodes=en2, elem_zone=np.zeros_like(m["elem_zone"]), ifaces_L=np.zeros((0, 2), np.int32),
              ifaces_R=np.zeros((0, 2), np.int32))
    for N in (3, 5):
        prm = FlowParams(omega=0.0)
        oa = oracle_mod.Oracle(m, N, prm)
        ob = oracle_mod.Oracle(m2, N, prm)
        Q = oa.state_from(lambda x, y: fields.isentropic_vortex(x, y, x0=1.0, y0=2.0))
        ra, rb = oa.residual(Q, 0.0), ob.residual(Q, 0.0)
        assert np.abs(ra - rb).max() < 5e-11 * np.abs(rb).max()
        prmv = FlowParams(omega=0.0, viscous=1, mu=0.02)
        oa = oracle_mod.Oracle(m, N, prmv)
        ob = oracle_mod.Oracle(m2, N, prmv)
        ra, rb = oa.residual(Q, 0.0), ob.residual(Q, 0.0)
        assert np.abs(ra - rb).max() < 5e-11 * np.abs(rb).max()


def _vortex_dqdt(x, y, omega, zone_rot):
    """Exact dQ/dt following the mesh: (V_g - U_inf) . grad Q (complex step)."""
    h = 1e-30
    fx = fields.isentropic_vortex(x + 1j * h, y).imag / h
    fy = fields.isentropic_vortex(x, y + 1j * h).imag / h
    ug = np.where(zone_rot, -omega * y, 0.0)
    vg = np.where(zone_rot, omega * x, 0.0)
    return (ug - 1.0)[..., None] * fx + vg[..., None] * fy


@pytest.mark.parametrize("N", [3, 4])
def test_vortex_truncation_error_converges(oracle_mod, N):
    # Sec. 4.1 vortex: the residual of the exact solution tends to its exact
    # time derivative at order >= N - 1 (the solution error is one order higher).
    errs = []
    omega = math.pi / 4
    for s in (2, 4):  # the scale-1 mesh (h = 1.25) under-resolves the vortex core
        m = small_rotor(s)
        o = oracle_mod.Oracle(m, N, FlowParams(omega=omega))
        x, y = o.sp_coords(0.0)
        Q = np.moveaxis(fields.isentropic_vortex(x, y), -1, 1).copy()
        R = o.residual(Q, 0.0)
        rot = (m["elem_zone"] == 1)[:, None, None] * np.ones_like(x, dtype=bool)
        ex = np.moveaxis(_vortex_dqdt(x, y, omega, rot), -1, 1)
        errs.append(np.abs(R - ex).max())
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert (rates > N - 1 - 0.25).all(), (errs, rates)


@pytest.mark.slow
@pytest.mark.parametrize("N", [3, 4])
def test_couette_truncation_error_converges(oracle_mod, N):
    # Sec. 4.2 Taylor-Couette: the residual of the exact steady state must tend
    # to its exact time derivative following the mesh at order >= N - 1 under
    # refinement, through walls, viscous fluxes and the viscous mortar
    # procedure.  Following a point of the rotating zone the scalars stay
    # constant but the Cartesian momentum turns: d(rho u, rho v)/dt =
    # omega d/dphi = -omega rho v_theta (x, y) / r.
    omega, mach, re = 1.0, 0.1, 10.0
    gamma, Tw = 1.4, 1.0
    Rgas = (omega / mach) ** 2 / (gamma * Tw)
    mu = omega / re
    prm = FlowParams(gamma=gamma, Rgas=Rgas, mu=mu, prandtl=0.72, omega=omega, viscous=1, T_wall=Tw)
    k = mu * gamma * Rgas / ((gamma - 1) * 0.72)
    ex = fields.CouetteExact(omega, 1.0, 2.0, mu, k, Rgas, Tw)
    errs = []
    for s in (1, 2, 4):
        m = meshes.couette_mesh(2 * s, 12 * s, 2 * s, 16 * s)
        o = oracle_mod.Oracle(m, N, prm)
        x, y = o.sp_coords(0.0)
        Q = np.moveaxis(ex.state(x, y), -1, 1).copy()
        R = o.residual(Q, 0.0)
        r = np.hypot(x, y)
        rot = (m["elem_zone"] == 1)[:, None, None]
        expect = np.zeros_like(R)
        expect[:, 1] = np.where(rot, -omega * Q[:, 0] * ex.v(r) * x / r, 0.0)
        expect[:, 2] = np.where(rot, -omega * Q[:, 0] * ex.v(r) * y / r, 0.0)
        errs.append(np.abs(R - expect).max())
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert (rates > N - 1 - 0.3).all(), (errs, rates)


def test_ssp_rk3_is_third_order_in_time(oracle_mod):
    # Sec. 3: explicit SSP Runge-Kutta; the three-stage scheme is third order:
    # halving dt divides the error at fixed final time by about 8.  A wrong
    # stage weight or stage time (which moves the mortars) drops the order.
    m = small_rotor()
    N = 3
    o = oracle_mod.Oracle(m, N, FlowParams(omega=1.3))
    Q0 = o.state_from(lambda x, y: fields.isentropic_vortex(x, y, x0=2.0))
    T = 0.016
    ref, _ = o.step(Q0, 0.0, T / 128, 128)
    errs = []
    for n in (2, 4, 8):
        q, t = o.step(Q0, 0.0, T / n, n)
        assert abs(t - T) < 1e-15
        errs.append(np.abs(q - ref).max())
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert (rates > 2.7).all(), (errs, rates)


def test_ssp_rk54_order_conditions(oracle_mod):
    # Sec. 4 uses a five-stage fourth-order SSP Runge-Kutta method; its
    # coefficients (not printed in the paper) must satisfy the eight Butcher
    # order conditions up to order four.
    A, b, c = oracle_mod.rk54_tableau()
    assert np.allclose(A.sum(axis=1), c, atol=1e-15)
    assert np.allclose(np.triu(A), 0.0)  # explicit
    conds = [
        (b.sum(), 1.0),
        (b @ c, 1 / 2),
        (b @ c ** 2, 1 / 3),
        (b @ (A @ c), 1 / 6),
        (b @ c ** 3, 1 / 4),
        (b @ (c * (A @ c)), 1 / 8),
        (b @ (A @ c ** 2), 1 / 12),
        (b @ (A @ (A @ c)), 1 / 24),
    ]
    for got, want in conds:
        assert abs(got - want) < 5e-14, (got, want)
    # SSP: all Shu-Osher weights are non-negative, i.e. b >= 0 and A >= 0
    assert (b >= 0).all() and (A >= -1e-15).all()


def test_ssp_rk54_is_fourth_order_in_time(oracle_mod):
    m = small_rotor()
    o = oracle_mod.Oracle(m, 3, FlowParams(omega=1.3))
    Q0 = o.state_from(lambda x, y: fields.isentropic_vortex(x, y, x0=2.0))
    T = 0.032
    ref, _ = o.step(Q0, 0.0, T / 64, 64, rk_stages=5)
    errs = []
    for n in (2, 4, 8):
        q, t = o.step(Q0, 0.0, T / n, n, rk_stages=5)
        assert abs(t - T) < 1e-15
        errs.append(np.abs(q - ref).max())
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert (rates > 3.6).all(), (errs, rates)
