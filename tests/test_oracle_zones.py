"""Oracle pins for several rotating zones (each with its own centre, angular
velocity and sliding interface; Sec. 2.2 per zone, Sec. 3.2 per interface).

The paper runs one rotating zone per case.  These pins fix what several
zones must give from facts that do not depend on the oracle: exact SD
derivatives of linear fields with each zone's own grid velocity, discrete
conservation through both interfaces, the half-turn symmetry of a symmetric
two-disk mesh, and a frozen aligned zone equal to the same cells joined
conformingly.
"""
import numpy as np
import pytest
from scipy.spatial import cKDTree

from helpers import face_kinds, neighbours_of, small_row, small_twin, sp_weights
from ssd_inputs import fields, meshes
from ssd_inputs.workloads import FlowParams


def test_twin_mesh_tables(oracle_mod):
    m = small_twin()
    z = m["elem_zone"]
    assert set(np.unique(z)) == {0, 1, 2}
    assert (z == 1).sum() == (z == 2).sum()
    for key, want in (("ifaces_L", 1), ("ifaces_R", 0)):
        assert (z[m[key][:, 0]] == want).all()
    z2 = m["zones"][0]
    assert (z[z2["ifaces_L"][:, 0]] == 2).all() and (z[z2["ifaces_R"][:, 0]] == 0).all()
    o = oracle_mod.Oracle(m, 3, FlowParams(omega=0.7))
    kind, nbr, rev = o.face_info()
    # every face classified: 4 * E faces, interface faces of both zones counted once
    n_if = sum(len(a) for a in (m["ifaces_L"], m["ifaces_R"], z2["ifaces_L"], z2["ifaces_R"]))
    assert (kind >= 0).all()
    assert ((kind == 3) | (kind == 4)).sum() == n_if
    # each interface's mortars split each of its faces exactly once
    for zone in (1, 2):
        mo = o.mortars(0.37, zone)
        zl = m if zone == 1 else z2
        nL, nR = len(zl["ifaces_L"]), len(zl["ifaces_R"])
        assert len(mo["lf"]) == nL + nR  # no node coincidences at this time
        for side, n in (("L", nL), ("R", nR)):
            sums = np.zeros(n)
            np.add.at(sums, mo["lf" if side == "L" else "rf"], mo["s" + side])
            np.testing.assert_allclose(sums, 1.0, atol=1e-13)


def test_bad_zone_meshes_are_rejected(oracle_mod):
    m = small_twin()
    bad = dict(m)
    z2 = dict(m["zones"][0])
    z2["ifaces_L"] = m["ifaces_L"]  # zone-1 cells listed as zone 2's rotating side
    bad["zones"] = [z2]
    with pytest.raises(ValueError):
        oracle_mod.Oracle(bad, 3, FlowParams())
    bad = dict(m)
    az = m["elem_arc_zone"].copy()
    az[np.flatnonzero(m["elem_zone"] == 2)[0]] = 1  # a zone-2 cell drawn about zone 1's centre
    bad["elem_arc_zone"] = az
    with pytest.raises(ValueError):
        oracle_mod.Oracle(bad, 3, FlowParams())
    bad = dict(m)
    ez = m["elem_zone"].copy()
    ez[0] = 3  # no zone 3
    bad["elem_zone"] = ez
    with pytest.raises(ValueError):
        oracle_mod.Oracle(bad, 3, FlowParams())


@pytest.mark.parametrize("N", [3, 4])
def test_linear_field_exact_with_each_zones_grid_velocity(oracle_mod, N):
    # Q linear in x and y with uniform velocity and pressure: every flux is
    # polynomial of low degree on straight cells, so the SD residual is exact:
    # dQ/dt = -((U - u_g) dQ/dx + (V - v_g) dQ/dy) with (u_g, v_g) =
    # omega_z x (r - c_z) of the cell's own zone.  A wrong centre or rate of
    # zone 2 changes (u_g, v_g) there.
    om1, om2, t, U, V, bx, by = 0.7, -0.45, 0.31, 0.4, -0.2, 0.05, -0.03
    m = meshes.perturb_nodes(small_twin(omega2=om2), 0.1, seed=5)
    o = oracle_mod.Oracle(m, N, FlowParams(omega=om1))
    x, y = o.sp_coords(t)
    rho = 1.0 + bx * x + by * y
    Q = np.moveaxis(fields.conservative(rho, U, V, np.full_like(x, 1.0)), -1, 1).copy()
    R = o.residual(Q, t)
    d = np.moveaxis(fields.conservative(np.full_like(x, 1.0), U, V, np.zeros_like(x)), -1, 1)
    d[:, 3] = 0.5 * (U * U + V * V)  # dQ/drho at fixed U, V, p
    zone = m["elem_zone"][:, None, None]
    cx = np.where(zone == 2, m["zones"][0]["center"][0], m["center"][0])
    cy = np.where(zone == 2, m["zones"][0]["center"][1], m["center"][1])
    om = np.select([zone == 1, zone == 2], [om1, om2], 0.0)
    ug, vg = -om * (y - cy), om * (x - cx)
    expect = -((U - ug) * bx + (V - vg) * by)[:, None] * d
    ok = ~neighbours_of(m, face_kinds(m) | _zone2_special(m))
    assert (m["elem_zone"][ok] == 1).sum() > 5 and (m["elem_zone"][ok] == 2).sum() > 5
    np.testing.assert_allclose(R[ok], expect[ok], atol=2e-13)


def _zone2_special(m):
    special = np.zeros(len(m["elem_nodes"]), dtype=bool)
    for key in ("ifaces_L", "ifaces_R"):
        special[m["zones"][0][key][:, 0]] = True
    return special


@pytest.mark.parametrize("N,viscous", [(3, 0), (4, 0), (4, 1)])
def test_discrete_conservation_through_two_interfaces(oracle_mod, N, viscous):
    # periodic box: sum_e sum_ij w_i w_j |J| dQ/dt = 0 for every variable, with
    # both zones turning at different rates and arbitrary mortar offsets
    m = small_twin(omega2=-0.6, shift_L=0.1234, shift_R=-0.05)
    prm = FlowParams(omega=0.9, viscous=viscous, mu=0.05 if viscous else 0.0)
    o = oracle_mod.Oracle(m, N, prm)
    Q = o.state_from(lambda x, y: fields.random_smooth_state(x, y, seed=11, amp=0.2, scale=3.0))
    R = o.residual(Q, 0.37)
    J = o.sp_jacobian()
    w = sp_weights(oracle_mod, N)
    total = np.einsum("evji,eji,j,i->v", R, J, w, w)
    scale = np.einsum("evji,eji,j,i->v", np.abs(R), J, w, w)
    assert (np.abs(total) < 1e-13 * scale).all(), total / scale


def _half_turn_state(x, y):
    # even density, pressure; odd velocity under (x, y) -> (-x, -y)
    rho = 1.0 + 0.1 * np.cos(0.7 * x) * np.cos(0.5 * y) + 0.05 * np.sin(0.3 * x) * np.sin(0.9 * y)
    u = 0.2 * np.sin(0.6 * x) * np.cos(0.4 * y) + 0.1 * np.sin(0.5 * y)
    v = 0.15 * np.sin(0.4 * x + 0.3 * y)
    p = 1.0 + 0.1 * np.cos(0.3 * x - 0.2 * y)
    return fields.conservative(rho, u, v, p)


@pytest.mark.parametrize("viscous", [0, 1])
def test_half_turn_symmetry_of_two_equal_zones(oracle_mod, viscous):
    # Disk 2 is the half turn of disk 1 about the origin and both turn at the
    # same rate, so the configuration is invariant under (x, y) -> (-x, -y):
    # for a state with even density / pressure and odd velocity, dQ/dt has the
    # same parity.  Every zone-2 quantity (centre, rate, interface angles,
    # mortar tables) is checked against its zone-1 counterpart.
    om, t = 0.8, 0.29
    m = small_twin(omega2=om, shift_L=0.07)
    prm = FlowParams(omega=om, viscous=viscous, mu=0.03 if viscous else 0.0)
    o = oracle_mod.Oracle(m, 4, prm)
    x, y = o.sp_coords(t)
    Q = np.ascontiguousarray(np.moveaxis(_half_turn_state(x, y), -1, 1))
    R = o.residual(Q, t)
    pts = np.stack([x.ravel(), y.ravel()], axis=1)
    dist, idx = cKDTree(pts).query(-pts)
    assert dist.max() < 1e-10
    Rf = np.moveaxis(R, 1, -1).reshape(-1, 4)
    sign = np.array([1.0, -1.0, -1.0, 1.0])
    scale = np.abs(Rf).max(axis=0)
    err = np.abs(Rf[idx] - sign * Rf).max(axis=0) / scale
    assert (err < 1e-10).all(), err
    # the two disks really are coupled through their own interfaces: zone 2's
    # residual is not zone 1's at the same local position
    assert np.abs(R).max() > 1e-3


def test_frozen_aligned_zone_equals_conforming_cells(oracle_mod):
    # Zone 2 with as many faces as its stationary side and omega_2 = 0: every
    # zone-2 mortar is a whole face (o = 0, s = 1), so its interface must equal
    # the same cells joined conformingly (zone 1 keeps turning in both runs).
    m = small_twin(omega2=0.0, n_core2=8)
    z2 = m["zones"][0]
    assert len(z2["ifaces_L"]) == len(z2["ifaces_R"])
    xy, en = m["xy"], m["elem_nodes"]
    Lnodes, Rnodes = set(), set()
    for key, acc in (("ifaces_L", Lnodes), ("ifaces_R", Rnodes)):
        for e, f in z2[key]:
            a, b = meshes.FACE_CORNERS[f]
            acc.update([en[e, a], en[e, b]])
    remap = {}
    for n in Lnodes:
        dist, r = min((np.hypot(*(xy[n] - xy[r])), r) for r in Rnodes)
        assert dist < 1e-12
        remap[n] = r
    m2 = dict(m)
    m2["elem_nodes"] = np.vectorize(lambda n: remap.get(n, n))(en).astype(np.int32)
    m2["elem_zone"] = np.where(m["elem_zone"] == 2, 0, m["elem_zone"]).astype(np.int32)
    m2["zones"] = [dict(z2, ifaces_L=np.zeros((0, 2), np.int32), ifaces_R=np.zeros((0, 2), np.int32))]
    for viscous in (0, 1):
        prm = FlowParams(omega=0.6, viscous=viscous, mu=0.02 if viscous else 0.0)
        oa = oracle_mod.Oracle(m, 4, prm)
        ob = oracle_mod.Oracle(m2, 4, prm)
        Q = oa.state_from(lambda x, y: fields.random_smooth_state(x, y, seed=3, amp=0.2, scale=2.0))
        ra, rb = oa.residual(Q, 0.21), ob.residual(Q, 0.21)
        assert np.abs(ra - rb).max() < 5e-11 * np.abs(rb).max()


def test_four_zones_conserve_and_a_fifth_is_rejected(oracle_mod):
    # the most rotating zones a mesh may have, each at its own rate and with
    # its own number of interface faces
    m = small_row(4, (-0.6, 0.3, 1.1), shift_L=0.1, n_cores=(4, 3, 5, 2))
    o = oracle_mod.Oracle(m, 3, FlowParams(omega=0.9))
    Q = o.state_from(lambda x, y: fields.random_smooth_state(x, y, seed=2, amp=0.2, scale=3.0))
    R = o.residual(Q, 0.41)
    J = o.sp_jacobian()
    w = sp_weights(oracle_mod, 3)
    total = np.einsum("evji,eji,j,i->v", R, J, w, w)
    scale = np.einsum("evji,eji,j,i->v", np.abs(R), J, w, w)
    assert (np.abs(total) < 1e-13 * scale).all(), total / scale
    for zone in (1, 2, 3, 4):
        assert len(o.mortars(0.41, zone)["lf"]) > 0
    with pytest.raises(ValueError):
        oracle_mod.Oracle(small_row(5, (-0.6, 0.3, 1.1, 0.2)), 3, FlowParams(omega=0.9))


def test_full_twin_rotor_workload_mesh(oracle_mod):
    # the two-zone bench workload: valid for the oracle (every face classified,
    # both interfaces closed), positive Jacobian at every SP, each interface's
    # mortars tiling its faces
    from ssd_inputs.workloads import build_workload
    w = build_workload("twin_rotor_n6")
    m = w.mesh
    assert len(m["elem_nodes"]) == 123450 and len(m["zones"]) == 1
    o = oracle_mod.Oracle(m, 3, w.params)
    assert (o.sp_jacobian() > 0).all()
    for zone in (1, 2):
        mo = o.mortars(0.37, zone)
        zl = m if zone == 1 else m["zones"][0]
        nL = len(zl["ifaces_L"])
        sums = np.zeros(nL)
        np.add.at(sums, mo["lf"], mo["sL"])
        np.testing.assert_allclose(sums, 1.0, atol=1e-13)
