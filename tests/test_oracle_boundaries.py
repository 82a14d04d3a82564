"""Pins of the oracle's 12-node cubic cells and of the boundary conditions of
the elliptic-cylinder case (Sec. 4: slip walls, Dirichlet inlet,
fixed-pressure outlet), against what geometry and conservation fix:

- a cell with cubic edges is the 12-node serendipity element, so a mapping in
  the serendipity span (x^a y^b, a + b <= 3, and x^3 y, x y^3) is reproduced
  exactly, positions and Jacobian;
- its metric terms are cubic in each direction, so for N >= 3 a uniform free
  stream is an exact discrete steady state on such cells, whatever the node
  positions;
- a slip wall passes no mass and (Euler) no energy: a closed slip box
  conserves both to round-off for any state;
- the outlet ghost keeps the interior density and velocity, so the mass
  leaving through it is exactly the integral of rho u . n, which is known in
  closed form for a polynomial state;
- the free-stream values enter only through the inlet and outlet faces;
- an adiabatic no-slip wall passes no mass and, at rest, no energy (no work,
  no heat), so a closed adiabatic box conserves both to round-off, viscous
  terms included, while an isothermal box exchanges heat; moving adiabatic
  walls (the stirred tank's blades) still pass no mass.
"""
import math

import numpy as np
import pytest

from helpers import sp_weights
from ssd_inputs import fields, meshes
from ssd_inputs.meshes import BC_ADIABATIC, BC_INLET, BC_OUTLET, BC_SLIP, BC_WALL
from ssd_inputs.workloads import FlowParams


def _in_span(x, y):
    # every term is in the cubic serendipity span
    return (x + 0.04 * y ** 3 + 0.02 * x * y - 0.01 * x ** 3 * y,
            y + 0.03 * x * x * y - 0.01 * x * y ** 3 + 0.05 * x * x)


def _out_of_span(x, y):
    return (x + 0.02 * x * x * y * y, y + 0.01 * x ** 3 * y * y)


def _span_jacobian(x, y):
    Xx = 1 + 0.02 * y - 0.03 * x * x * y
    Xy = 0.12 * y * y + 0.02 * x - 0.01 * x ** 3
    Yx = 0.06 * x * y - 0.01 * y ** 3 + 0.1 * x
    Yy = 1 + 0.03 * x * x - 0.03 * x * y * y
    return Xx * Yy - Xy * Yx


def _free_stream_params(viscous=0):
    return FlowParams(gamma=1.4, Rgas=1.0, mu=0.02 if viscous else 0.0, viscous=viscous, rho_inf=1.1,
                      u_inf=0.6, v_inf=-0.25, p_inf=0.9)


@pytest.mark.parametrize("N", [3, 4, 5])
def test_cubic_cells_reproduce_serendipity_map(oracle_mod, N):
    nx, ny, lx, ly = 3, 2, 3.0, 2.0
    m = meshes.channel_mesh(nx, ny, lx, ly, tags=(BC_INLET,) * 4, mapping=_in_span, cubic=True)
    o = oracle_mod.Oracle(m, N, _free_stream_params())
    Xs, _ = oracle_mod.points(N)
    X, Y = o.sp_coords()
    J = o.sp_jacobian()
    hx, hy = lx / nx, ly / ny
    for e in range(nx * ny):
        i, j = e % nx, e // nx
        xs = (i + Xs[None, :]) * hx + 0 * Xs[:, None]
        ys = (j + Xs[:, None]) * hy + 0 * Xs[None, :]
        Xe, Ye = _in_span(xs, ys)
        np.testing.assert_allclose(X[e], Xe, rtol=0, atol=1e-14)
        np.testing.assert_allclose(Y[e], Ye, rtol=0, atol=1e-14)
        np.testing.assert_allclose(J[e], _span_jacobian(xs, ys) * hx * hy, rtol=1e-13, atol=0)


def test_out_of_span_map_is_not_reproduced(oracle_mod):
    # control for the test above: a quartic term is only interpolated
    m = meshes.channel_mesh(3, 2, 3.0, 2.0, tags=(BC_INLET,) * 4, mapping=_out_of_span, cubic=True)
    o = oracle_mod.Oracle(m, 4, _free_stream_params())
    Xs, _ = oracle_mod.points(4)
    X, _ = o.sp_coords()
    xs = Xs[None, :] + 0 * Xs[:, None]
    ys = Xs[:, None] + 0 * Xs[None, :]
    assert np.abs(X[0] - _out_of_span(xs, ys)[0]).max() > 1e-6


@pytest.mark.parametrize("N", [3, 4, 5])
@pytest.mark.parametrize("viscous", [0, 1])
@pytest.mark.parametrize("mapping", [_in_span, _out_of_span])
def test_free_stream_on_cubic_cells(oracle_mod, N, viscous, mapping):
    prm = _free_stream_params(viscous)
    m = meshes.channel_mesh(3, 2, 3.0, 2.0, tags=(BC_INLET,) * 4, mapping=mapping, cubic=True)
    o = oracle_mod.Oracle(m, N, prm)
    Q = o.state_from(lambda x, y: fields.uniform(x, y, rho=prm.rho_inf, u=prm.u_inf, v=prm.v_inf,
                                                 p=prm.p_inf))
    R, S = o.residual_with_scale(Q, 0.0)
    assert np.abs(R).max() < 1e-13 * S.max() * N * N, np.abs(R).max()


@pytest.mark.parametrize("N", [3, 5])
@pytest.mark.parametrize("cubic", [False, True])
def test_closed_slip_box_conserves_mass_and_energy(oracle_mod, N, cubic):
    m = meshes.channel_mesh(4, 3, 3.0, 2.0, tags=(BC_SLIP,) * 4, mapping=_in_span if cubic else None,
                            cubic=cubic)
    o = oracle_mod.Oracle(m, N, _free_stream_params())
    Q = o.state_from(lambda x, y: fields.random_smooth_state(x, y, seed=7, amp=0.2, scale=1.5))
    R = o.residual(Q, 0.0)
    J = o.sp_jacobian()
    w = sp_weights(oracle_mod, N)
    total = np.einsum("evji,eji,j,i->v", R, J, w, w)
    scale = np.einsum("evji,eji,j,i->v", np.abs(R), J, w, w)
    assert abs(total[0]) < 1e-13 * scale[0] and abs(total[3]) < 1e-13 * scale[3], total / scale
    # the walls do exert a pressure force: momentum is not conserved
    assert abs(total[1]) > 1e-6 * scale[1]


def test_closed_slip_box_viscous_conserves_mass(oracle_mod):
    m = meshes.channel_mesh(4, 3, 3.0, 2.0, tags=(BC_SLIP,) * 4, mapping=_in_span, cubic=True)
    o = oracle_mod.Oracle(m, 4, _free_stream_params(viscous=1))
    Q = o.state_from(lambda x, y: fields.random_smooth_state(x, y, seed=8, amp=0.2, scale=1.5))
    R = o.residual(Q, 0.0)
    total = np.einsum("evji,eji,j,i->v", R, o.sp_jacobian(), *(2 * [sp_weights(oracle_mod, 4)]))
    scale = np.einsum("evji,eji,j,i->v", np.abs(R), o.sp_jacobian(), *(2 * [sp_weights(oracle_mod, 4)]))
    assert abs(total[0]) < 1e-13 * scale[0]


@pytest.mark.parametrize("N", [3, 4])
@pytest.mark.parametrize("viscous", [0, 1])
def test_outlet_mass_flux_closed_form(oracle_mod, N, viscous):
    # slip walls left, bottom, top; outlet at x = lx.  For a state whose
    # conservative variables are polynomials of degree <= N - 1 the face
    # traces are exact, so d/dt (total mass) = - int_0^ly (rho u)(lx, y) dy.
    lx, ly = 3.0, 2.0
    m = meshes.channel_mesh(4, 3, lx, ly, tags=(BC_SLIP, BC_OUTLET, BC_SLIP, BC_SLIP))
    prm = _free_stream_params(viscous)

    def state(x, y):
        rho = 1.0 + 0.1 * x + 0.05 * y
        mx = 0.3 + 0.1 * y - 0.05 * x * y
        my = 0.02 * x
        E = 2.5 + 0.1 * y
        return np.stack([rho, mx, my + 0 * x, E + 0 * x], axis=-1)

    o = oracle_mod.Oracle(m, N, prm)
    Q = o.state_from(state)
    R = o.residual(Q, 0.0)
    w = sp_weights(oracle_mod, N)
    total = np.einsum("eji,eji,j,i->", R[:, 0], o.sp_jacobian(), w, w)
    # int_0^ly (0.3 + 0.1 y - 0.05 lx y) dy
    exact = 0.3 * ly + (0.1 - 0.05 * lx) * ly * ly / 2.0
    assert abs(total + exact) < 1e-13, (total, exact)


def _adjacent(m, tag):
    return {int(e) for e, f, t in m["bfaces"] if t == tag}


@pytest.mark.parametrize("field", ["rho_inf", "u_inf", "v_inf", "p_inf"])
def test_free_stream_enters_only_at_inlet_and_outlet(oracle_mod, field):
    m = meshes.channel_mesh(5, 3, 3.0, 2.0, tags=(BC_INLET, BC_OUTLET, BC_SLIP, BC_SLIP))
    prm = _free_stream_params()
    Qf = lambda x, y: fields.random_smooth_state(x, y, seed=3, amp=0.1, scale=1.5)
    o = oracle_mod.Oracle(m, 4, prm)
    R0 = o.residual(o.state_from(Qf), 0.0)
    prm2 = _free_stream_params()
    setattr(prm2, field, getattr(prm2, field) + 0.1)
    o2 = oracle_mod.Oracle(m, 4, prm2)
    R1 = o2.residual(o2.state_from(Qf), 0.0)
    changed = {int(e) for e in np.where(np.abs(R1 - R0).max(axis=(1, 2, 3)) > 0)[0]}
    expect = _adjacent(m, BC_INLET) | (_adjacent(m, BC_OUTLET) if field == "p_inf" else set())
    assert changed == expect


def test_bad_curved_meshes_are_rejected(oracle_mod):
    m = meshes.channel_mesh(3, 2, 3.0, 2.0, tags=(BC_INLET,) * 4, mapping=_in_span, cubic=True)
    prm = _free_stream_params()
    bad = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in m.items()}
    # the two cells sharing a face disagree on its edge nodes
    e0_f1 = bad["edge_nodes"][0, 1].copy()
    bad["edge_nodes"][0, 1] = e0_f1[::-1]
    with pytest.raises(ValueError, match="cubic edge nodes"):
        oracle_mod.Oracle(bad, 3, prm)
    bad = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in m.items()}
    bad["edge_arc"][0, 1] = 0  # straight on one side, cubic on the other
    with pytest.raises(ValueError, match="edge kinds differ"):
        oracle_mod.Oracle(bad, 3, prm)
    bad = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in m.items()}
    bad["bfaces"][0, 2] = 9
    with pytest.raises(ValueError, match="boundary tag"):
        oracle_mod.Oracle(bad, 3, prm)


def test_ellipse_mesh_is_valid(oracle_mod):
    m = meshes.ellipse_mesh(n_theta=32, n_inner=6, n_outer=8)
    st = meshes.mesh_stats(m)
    assert st["interface_L"] == st["interface_R"] == 32
    tags = np.bincount(m["bfaces"][:, 2], minlength=5)
    assert tags[BC_WALL] == 32 and tags[BC_INLET] > 0 and tags[BC_OUTLET] > 0 and tags[BC_SLIP] > 0
    o = oracle_mod.Oracle(m, 5, _free_stream_params())
    assert o.sp_jacobian().min() > 0
    # the cubic edges on the body follow the ellipse to the interpolation error
    x, y = o.sp_coords()
    body = [int(e) for e, f, t in m["bfaces"] if t == BC_WALL]
    r_body = np.hypot(x[body] / 0.5, y[body] / 0.1)
    assert r_body.min() > 1.0  # the SPs lie outside the ellipse


def _closed_box_totals(oracle_mod, tag, N=4, zone=0, omega=0.0, seed=12):
    m = meshes.channel_mesh(4, 3, 3.0, 2.0, tags=(tag,) * 4, mapping=_in_span, cubic=True, zone=zone)
    prm = FlowParams(gamma=1.4, Rgas=1.0, mu=0.05, viscous=1, T_wall=1.3, omega=omega)
    o = oracle_mod.Oracle(m, N, prm)
    Q = o.state_from(lambda x, y: fields.random_smooth_state(x, y, seed=seed, amp=0.2, scale=1.5))
    R = o.residual(Q, 0.3)
    w = sp_weights(oracle_mod, N)
    J = o.sp_jacobian()
    total = np.einsum("evji,eji,j,i->v", R, J, w, w)
    scale = np.einsum("evji,eji,j,i->v", np.abs(R), J, w, w)
    return total / scale


@pytest.mark.parametrize("N", [3, 5])
def test_closed_adiabatic_box_conserves_mass_and_energy(oracle_mod, N):
    rel = _closed_box_totals(oracle_mod, BC_ADIABATIC, N)
    assert abs(rel[0]) < 1e-13 and abs(rel[3]) < 1e-13, rel


def test_closed_isothermal_box_exchanges_heat(oracle_mod):
    # control: the same box with isothermal walls at a different temperature
    rel = _closed_box_totals(oracle_mod, BC_WALL)
    assert abs(rel[3]) > 1e-6, rel


def test_moving_adiabatic_walls_pass_no_mass(oracle_mod):
    # the whole box rotates; its walls move normal to themselves
    rel = _closed_box_totals(oracle_mod, BC_ADIABATIC, zone=1, omega=0.8)
    assert abs(rel[0]) < 1e-13, rel
    assert abs(rel[3]) > 1e-6  # moving walls do work


def test_stirred_tank_mesh_is_valid(oracle_mod):
    m = meshes.stirred_tank_mesh(n_theta_in=48, n_theta_out=40, layers_in=(3, 4, 3), layers_out=(3, 4))
    tags = np.bincount(m["bfaces"][:, 2], minlength=6)
    # 6 blades x (2 x 4 long faces + 2 x 2 end faces) adiabatic
    assert tags[BC_ADIABATIC] == 6 * (2 * 4 + 4)
    o = oracle_mod.Oracle(m, 4, FlowParams(omega=1.0, viscous=1, mu=0.01, Rgas=25 / 1.4))
    assert o.sp_jacobian().min() > 0
    # blades are exact rectangles: every adiabatic face point lies on a plate face
    x, y = o.sp_coords()
    for e, f, t in m["bfaces"]:
        if t != BC_ADIABATIC:
            continue
        xe, ye = x[e].mean(), y[e].mean()
        th = round(math.atan2(ye, xe) / (2 * math.pi / 6)) * (2 * math.pi / 6)
        en = m["elem_nodes"][e]
        i, j = meshes.FACE_CORNERS[f]
        for n in (en[i], en[j]):
            along = m["xy"][n, 0] * math.cos(th) + m["xy"][n, 1] * math.sin(th)
            perp = -m["xy"][n, 0] * math.sin(th) + m["xy"][n, 1] * math.cos(th)
            assert (abs(abs(perp) - 0.05) < 1e-12 and 1.0 - 1e-12 <= along <= 2.0 + 1e-12) or \
                (abs(perp) <= 0.05 + 1e-12 and min(abs(along - 1.0), abs(along - 2.0)) < 1e-12)
