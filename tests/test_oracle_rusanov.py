"""Pins of the oracle's Rusanov common flux (Sec. 3.1) and of how the residual
uses it on faces with jumps.

The smooth-state pins elsewhere hold for any wave speed: a continuous state
has no jump at a face, so the dissipation term of the common flux vanishes
there.  These pins use states that jump across faces:

  * the flux itself against hand-derived golden values (tests/golden/
    rusanov_flux.json): a stationary subsonic and a supersonic jump, and two
    moving faces whose wave speed changes when the grid velocity is left out;
  * the residual of a two-state stripe on a periodic box: with a constant
    state per cell the interior flux polynomial has zero divergence on
    straight cells, so each solution point's residual is the end flux-point
    corrections alone, -(1/|J|) (l'_0 dF_left + l'_N dF_right), with the golden
    common fluxes and the flux-point basis derivatives evaluated here with
    numpy;
  * the same closed form on every straight cell of a rotor mesh with a random
    constant state per cell at a rotated position, where the conforming faces
    of the rotating zone move (V_g . n != 0).
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from helpers import random_cell_states, small_rotor, small_twin
from ssd_inputs import meshes
from ssd_inputs.workloads import FlowParams

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "rusanov_flux.json")
FACE_CORNERS = ((0, 1), (1, 2), (3, 2), (0, 3))  # local face f: start and end corner of its parameter
FACE_SIGN = (-1.0, 1.0, 1.0, -1.0)               # F~_end = sign_f |a_f| F . n_out


def _golden():
    with open(GOLDEN) as f:
        return json.load(f)


def conservative(prim, gamma):
    rho, u, v, p = prim
    return np.array([rho, rho * u, rho * v, p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)])


def normal_flux(q, n, vgn, gamma):
    """F(Q).n - v_gn Q (Sec. 2.1 Euler fluxes with the grid-velocity term of Sec. 2.2)."""
    rho, mu, mv, E = q
    p = (gamma - 1.0) * (E - 0.5 * (mu * mu + mv * mv) / rho)
    un = (mu * n[0] + mv * n[1]) / rho
    return np.array([rho * un, mu * un + p * n[0], mv * un + p * n[1], (E + p) * un]) - vgn * np.asarray(q)


def sd_points(N):
    """Solution points (Chebyshev-Gauss on [0,1]) and flux points (0, the
    N-1 Legendre-Gauss points, 1), Sec. 3.1, from numpy."""
    s = np.arange(1, N + 1)
    Xs = 0.5 * (1.0 - np.cos((2 * s - 1) * np.pi / (2 * N)))
    z, _ = np.polynomial.legendre.leggauss(N - 1)
    Xf = np.concatenate([[0.0], 0.5 * (1.0 + np.sort(z)), [1.0]])
    return Xs, Xf


def fp_basis_derivative(N):
    """D[k, i] = l'_i(X_k): derivative of the flux-point Lagrange basis
    (degree N) at the solution points, by numpy polynomial products."""
    Xs, Xf = sd_points(N)
    D = np.zeros((N, N + 1))
    for i in range(N + 1):
        others = np.delete(Xf, i)
        P = np.polynomial.Polynomial.fromroots(others) / np.prod(Xf[i] - others)
        D[:, i] = P.deriv()(Xs)
    return D


# ---------------------------------------------------------------------------
# the flux against hand-derived values
# ---------------------------------------------------------------------------

def test_golden_file_is_self_consistent():
    # the stored fractions satisfy the stated definition exactly (guards the
    # file against typing slips; the oracle is not involved)
    g = _golden()
    gam = Fraction(g["gamma"]).limit_denominator(10)
    for c in g["cases"]:
        def cons(prim):
            rho, u, v, p = (Fraction(x).limit_denominator(1000) for x in prim)
            return [rho, rho * u, rho * v, p / (gam - 1) + Fraction(1, 2) * rho * (u * u + v * v)], p, u, v, rho
        (qL, pL, uL, vL, rL), (qR, pR, uR, vR, rR) = cons(c["prim_L"]), cons(c["prim_R"])
        n = [Fraction(x).limit_denominator(10) for x in c["n"]]
        vgn = Fraction(c["vgn"]).limit_denominator(10)
        cs = [Fraction(x) for x in c["c"]]
        assert cs[0] ** 2 == gam * pL / rL and cs[1] ** 2 == gam * pR / rR
        lam = max(abs(uL * n[0] + vL * n[1] - vgn) + cs[0], abs(uR * n[0] + vR * n[1] - vgn) + cs[1])
        assert lam == Fraction(c["lambda"])

        def fn(q, p):
            un = (q[1] * n[0] + q[2] * n[1]) / q[0]
            return [q[0] * un - vgn * q[0], q[1] * un + p * n[0] - vgn * q[1], q[2] * un + p * n[1] - vgn * q[2],
                    (q[3] + p) * un - vgn * q[3]]
        fL, fR = fn(qL, pL), fn(qR, pR)
        if "Fn_L" in c:
            assert [Fraction(x) for x in c["Fn_L"]] == fL and [Fraction(x) for x in c["Fn_R"]] == fR
        F = [Fraction(1, 2) * (a + b) - Fraction(1, 2) * lam * (r - l) for a, b, l, r in zip(fL, fR, qL, qR)]
        assert [Fraction(x) for x in c["F_common"]] == F
        assert np.allclose([float(x) for x in F], c["F_common_decimal"], rtol=0, atol=1e-15)


@pytest.mark.parametrize("case", [c["name"] for c in _golden()["cases"]])
def test_rusanov_matches_golden(oracle_mod, case):
    g = _golden()
    c = next(x for x in g["cases"] if x["name"] == case)
    qL, qR = conservative(c["prim_L"], g["gamma"]), conservative(c["prim_R"], g["gamma"])
    F = oracle_mod.rusanov(g["gamma"], qL, qR, c["n"], c["vgn"])
    np.testing.assert_allclose(F, c["F_common_decimal"], rtol=2e-15, atol=2e-15)


def test_rusanov_consistency_and_antisymmetry(oracle_mod):
    rng = np.random.Generator(np.random.PCG64(11))
    for _ in range(20):
        gam = 1.4
        a = conservative([rng.uniform(0.3, 2), *rng.uniform(-1, 1, 2), rng.uniform(0.3, 2)], gam)
        b = conservative([rng.uniform(0.3, 2), *rng.uniform(-1, 1, 2), rng.uniform(0.3, 2)], gam)
        phi = rng.uniform(0, 2 * math.pi)
        n = (math.cos(phi), math.sin(phi))
        vgn = rng.uniform(-1, 1)
        # equal states: the physical normal flux, exactly
        assert np.array_equal(oracle_mod.rusanov(gam, a, a, n, vgn), normal_flux(a, n, vgn, gam)) or \
            np.allclose(oracle_mod.rusanov(gam, a, a, n, vgn), normal_flux(a, n, vgn, gam), rtol=1e-15, atol=1e-15)
        # seen from the other side (normal and grid velocity reversed) the flux changes sign
        f1 = oracle_mod.rusanov(gam, a, b, n, vgn)
        f2 = oracle_mod.rusanov(gam, b, a, (-n[0], -n[1]), -vgn)
        np.testing.assert_allclose(f2, -f1, rtol=1e-15, atol=1e-15)


# ---------------------------------------------------------------------------
# the residual on piecewise-constant states
# ---------------------------------------------------------------------------

def _cell_index_of_columns(o, mesh):
    x, _ = o.sp_coords(0.0)
    return x.mean(axis=(1, 2))


@pytest.mark.parametrize("N", [3, 4, 5])
def test_two_state_stripe_residual(oracle_mod, N):
    # periodic 2 x 2 box of unit squares: the left column holds state A, the
    # right column state B (case A of the golden file).  The x-faces carry the
    # golden common fluxes F(A|B) at x = 0 and F(B|A) at x = +-1; the y-faces
    # join equal states.  Per cell: R(i, j) = -(1/h) [l'_0(X_i) (F_left - F_x(Q))
    # + l'_N(X_i) (F_right - F_x(Q))], independent of j.
    g = _golden()
    gam = g["gamma"]
    cA = next(c for c in g["cases"] if c["name"] == "A_stationary_subsonic")
    cB = next(c for c in g["cases"] if c["name"] == "A_reversed")
    qA, qB = conservative(cA["prim_L"], gam), conservative(cA["prim_R"], gam)
    F_AB, F_BA = np.array(cA["F_common_decimal"]), np.array(cB["F_common_decimal"])
    FxA = np.array([float(Fraction(x)) for x in cA["Fn_L"]])
    FxB = np.array([float(Fraction(x)) for x in cA["Fn_R"]])
    m = meshes.periodic_box_mesh(2, 1.0)
    o = oracle_mod.Oracle(m, N, FlowParams(gamma=gam))
    xc = _cell_index_of_columns(o, m)
    Q = np.zeros(o.shape)
    left = xc < 0
    Q[left] = qA[None, :, None, None]
    Q[~left] = qB[None, :, None, None]
    R = o.residual(Q, 0.0)
    D = fp_basis_derivative(N)
    h = 1.0
    expA = -(np.outer(F_BA - FxA, D[:, 0]) + np.outer(F_AB - FxA, D[:, N])) / h   # [v][i]
    expB = -(np.outer(F_AB - FxB, D[:, 0]) + np.outer(F_BA - FxB, D[:, N])) / h
    scale = max(np.abs(expA).max(), np.abs(expB).max())
    for e in range(o.E):
        exp = expA if left[e] else expB
        np.testing.assert_allclose(R[e], np.broadcast_to(exp[:, None, :], (4, N, N)), rtol=0, atol=5e-14 * scale)


def _face_neighbours(mesh):
    """(e, f) -> (e', f') across conforming faces (shared node pair) and
    periodic pairs, from the mesh arrays."""
    en = mesh["elem_nodes"]
    open_, nb = {}, {}
    special = set()
    for key in ("ifaces_L", "ifaces_R"):
        for e, f in np.asarray(mesh[key]).reshape(-1, 2):
            special.add((int(e), int(f)))
    for z in mesh.get("zones", []):
        for key in ("ifaces_L", "ifaces_R"):
            for e, f in np.asarray(z[key]).reshape(-1, 2):
                special.add((int(e), int(f)))
    for row in mesh["bfaces"]:
        special.add((int(row[0]), int(row[1])))
    for row in mesh["pfaces"]:
        a, b = (int(row[0]), int(row[1])), (int(row[2]), int(row[3]))
        nb[a], nb[b] = b, a
        special.update((a, b))
    for e in range(len(en)):
        for f, (i, j) in enumerate(FACE_CORNERS):
            if (e, f) in special:
                continue
            key = (min(en[e, i], en[e, j]), max(en[e, i], en[e, j]))
            if key in open_:
                o = open_.pop(key)
                nb[o], nb[(e, f)] = (e, f), o
            else:
                open_[key] = (e, f)
    return nb


def expected_piecewise_constant(mesh, N, gamma, Qc, t, rusanov, zone_rates):
    """Residual of a state that is constant in each cell (Qc[e]), at every
    straight cell whose four faces are conforming or periodic: only the end
    flux-point corrections remain (the interior divergence of a constant state
    vanishes on straight cells, grid-velocity terms included).  Geometry of the
    bilinear map and the grid velocity omega x (x - c) of each rotating zone
    at angle omega t are evaluated here; the common flux is ``rusanov``.
    Returns (mask of checked cells, expected R)."""
    xy, en, arc, zone = mesh["xy"], mesh["elem_nodes"], mesh["edge_arc"], mesh["elem_zone"]
    nb = _face_neighbours(mesh)
    Xs, _ = sd_points(N)
    D = fp_basis_derivative(N)
    E = len(en)
    mask = np.zeros(E, dtype=bool)
    R = np.zeros((E, 4, N, N))
    for e in range(E):
        if arc[e].any() or not all((e, f) in nb for f in range(4)):
            continue
        z = int(zone[e])
        c = np.array(xy[en[e]], dtype=np.float64)
        if z:
            cx, cy, om = zone_rates[z]
            th = om * t
            cs, sn = math.cos(th), math.sin(th)
            d = c - [cx, cy]
            c = np.stack([cx + cs * d[:, 0] - sn * d[:, 1], cy + sn * d[:, 0] + cs * d[:, 1]], axis=1)
        e1, e3, dd = c[1] - c[0], c[3] - c[0], c[2] - c[1] - c[3] + c[0]

        def geo(xi, eta):
            x = c[0] + xi * e1 + eta * e3 + xi * eta * dd
            x_xi, x_eta = e1 + eta * dd, e3 + xi * dd
            return x, x_xi, x_eta

        dF = np.zeros((4, N, 4))  # [face][point][var]
        for f in range(4):
            en2 = nb[(e, f)][0]
            for j in range(N):
                xi, eta = {0: (Xs[j], 0.0), 1: (1.0, Xs[j]), 2: (Xs[j], 1.0), 3: (0.0, Xs[j])}[f]
                x, x_xi, x_eta = geo(xi, eta)
                a = np.array([x_eta[1], -x_eta[0]]) if f in (1, 3) else np.array([-x_xi[1], x_xi[0]])
                S = np.hypot(*a)
                n = FACE_SIGN[f] * a / S
                vgn = 0.0
                if z:
                    cx, cy, om = zone_rates[z]
                    vgn = om * (-(x[1] - cy) * n[0] + (x[0] - cx) * n[1])
                Fc = rusanov(gamma, Qc[e], Qc[en2], n, vgn)
                dF[f, j] = FACE_SIGN[f] * S * (Fc - normal_flux(Qc[e], n, vgn, gamma))
        for j in range(N):
            for i in range(N):
                _, x_xi, x_eta = geo(Xs[i], Xs[j])
                J = x_xi[0] * x_eta[1] - x_eta[0] * x_xi[1]
                div = D[i, 0] * dF[3, j] + D[i, N] * dF[1, j] + D[j, 0] * dF[0, i] + D[j, N] * dF[2, i]
                R[e, :, j, i] = -div / J
        mask[e] = True
    return mask, R


def zone_rates_of(mesh, omega):
    out = {1: (float(mesh["center"][0]), float(mesh["center"][1]), omega)}
    for k, z in enumerate(mesh.get("zones", [])):
        out[k + 2] = (float(z["center"][0]), float(z["center"][1]), float(z["omega"]))
    return out


@pytest.mark.parametrize("N", [3, 4])
@pytest.mark.parametrize("which", ["rotor", "twin"])
def test_piecewise_constant_residual_on_moving_faces(oracle_mod, N, which):
    mesh = meshes.perturb_nodes(small_rotor(shift_R=0.05), 0.15, seed=5) if which == "rotor" else small_twin()
    omega, t = 0.9, 0.77
    prm = FlowParams(omega=omega)
    o = oracle_mod.Oracle(mesh, N, prm)
    E = o.E
    Qc = random_cell_states(E, seed=N + 17)
    Q = np.ascontiguousarray(np.broadcast_to(Qc[:, :, None, None], (E, 4, N, N)))
    R = o.residual(Q, t)
    mask, Rexp = expected_piecewise_constant(mesh, N, prm.gamma, Qc, t, oracle_mod.rusanov,
                                             zone_rates_of(mesh, omega))
    zone = np.asarray(mesh["elem_zone"])
    assert mask[zone > 0].sum() >= 8 and mask[zone == 0].sum() >= 8  # moving and fixed faces both covered
    scale = np.abs(Rexp[mask]).max()
    np.testing.assert_allclose(R[mask], Rexp[mask], rtol=0, atol=1e-12 * scale)
