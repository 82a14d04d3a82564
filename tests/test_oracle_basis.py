"""Pins of the oracle's basis and mortar projections (Secs. 3.1, 3.2)."""
import numpy as np
import pytest
from numpy.polynomial import chebyshev, legendre
from scipy import integrate

NS = [2, 3, 4, 5, 6, 7]


@pytest.mark.parametrize("N", NS)
def test_solution_points_are_chebyshev_gauss(oracle_mod, N):
    # Sec. 3.1: SPs are the N Chebyshev-Gauss points, i.e. the roots of T_N mapped to [0,1]
    Xs, _ = oracle_mod.points(N)
    roots = np.sort(chebyshev.chebroots([0] * N + [1]))
    np.testing.assert_allclose(Xs, 0.5 * (1 + roots), rtol=0, atol=1e-15)
    assert np.all(np.diff(Xs) > 0)


@pytest.mark.parametrize("N", NS)
def test_flux_points_are_legendre_gauss_plus_ends(oracle_mod, N):
    # Sec. 3.1: FPs are the N-1 Legendre-Gauss points plus both end points
    _, Xf = oracle_mod.points(N)
    z, _ = legendre.leggauss(N - 1)
    assert Xf[0] == 0.0 and Xf[-1] == 1.0
    np.testing.assert_allclose(Xf[1:-1], 0.5 * (1 + z), rtol=0, atol=1e-15)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 9])
def test_gauss_legendre_matches_numpy(oracle_mod, n):
    x, w = oracle_mod.gauss_legendre(n)
    xr, wr = legendre.leggauss(n)
    np.testing.assert_allclose(x, xr, atol=2e-16)
    np.testing.assert_allclose(w, wr, atol=4e-16)


@pytest.mark.parametrize("N", NS)
def test_lagrange_bases(oracle_mod, N):
    # Eqs. hbasis / lbasis: cardinal property, partition of unity, exact derivatives
    Xs, Xf = oracle_mod.points(N)
    x = np.linspace(-0.1, 1.1, 37)
    for nodes in (Xs, Xf):
        n = len(nodes)
        val, der = oracle_mod.lagrange(nodes, nodes)
        np.testing.assert_allclose(val, np.eye(n), atol=1e-14)
        val, der = oracle_mod.lagrange(nodes, x)
        np.testing.assert_allclose(val.sum(axis=1), 1.0, atol=1e-13)
        np.testing.assert_allclose(der.sum(axis=1), 0.0, atol=1e-11)
        for p in range(n):
            np.testing.assert_allclose(val @ nodes ** p, x ** p, atol=1e-12)
            if p >= 1:
                np.testing.assert_allclose(der @ nodes ** p, p * x ** (p - 1), atol=1e-10)


def _l2_projection_by_quad(oracle_mod, N, o, s):
    """Unweighted L2 projection of Eq. prjQ1 solved from Gram matrices that
    scipy's adaptive quadrature integrates (independent of the oracle's rule)."""
    Xs, _ = oracle_mod.points(N)

    def h(i, x):
        v, _ = oracle_mod.lagrange(Xs, np.atleast_1d(x))
        return v[:, i]

    M = np.zeros((N, N))
    S = np.zeros((N, N))
    for i in range(N):
        for j in range(N):
            M[i, j] = integrate.quad(lambda z: h(i, z)[0] * h(j, z)[0], 0, 1, epsabs=1e-15)[0]
            S[i, j] = integrate.quad(lambda z: h(i, o + s * z)[0] * h(j, z)[0], 0, 1, epsabs=1e-15)[0]
    return np.linalg.solve(M, S.T), s * np.linalg.solve(M, S)


@pytest.mark.parametrize("N", [3, 4, 6])
@pytest.mark.parametrize("o,s", [(0.0, 1.0), (0.0, 0.37), (0.37, 0.63), (0.2, 0.5), (0.9, 0.1)])
def test_projection_matches_adaptive_quadrature(oracle_mod, N, o, s):
    Pf, Pb = oracle_mod.projection(N, o, s)
    Pf2, Pb2 = _l2_projection_by_quad(oracle_mod, N, o, s)
    np.testing.assert_allclose(Pf, Pf2, atol=1e-11)
    np.testing.assert_allclose(Pb, Pb2, atol=1e-11)


@pytest.mark.parametrize("N", NS)
def test_projection_identities(oracle_mod, N):
    rng = np.random.default_rng(7)
    Xs, _ = oracle_mod.points(N)
    # o = 0, s = 1: both projections are the identity
    Pf, Pb = oracle_mod.projection(N, 0.0, 1.0)
    np.testing.assert_allclose(Pf, np.eye(N), atol=1e-13)
    np.testing.assert_allclose(Pb, np.eye(N), atol=1e-13)
    # a face split into mortars at random break points
    cuts = np.sort(np.concatenate([[0.0, 1.0], rng.uniform(0, 1, 3)]))
    coef = rng.standard_normal(N)
    poly = lambda x: np.polyval(coef, x)
    face = poly(Xs)
    acc = np.zeros((N, N))
    w = _weights(oracle_mod, N)
    back = np.zeros(N)
    for a, b in zip(cuts[:-1], cuts[1:]):
        o, s = a, b - a
        Pf, Pb = oracle_mod.projection(N, o, s)
        # polynomial reproduction: degree N-1 data restricted to the mortar is exact
        np.testing.assert_allclose(Pf @ face, poly(o + s * Xs), atol=1e-11)
        acc += Pb @ Pf
        g = rng.standard_normal(N)
        back += Pb @ g
        # integral preservation: int_face (P_b g) = s int_mortar g
        np.testing.assert_allclose(w @ (Pb @ g), s * (w @ g), atol=1e-13)
    # projecting to the mortars and back recovers the face polynomial
    np.testing.assert_allclose(acc, np.eye(N), atol=1e-11)


def _weights(oracle_mod, N):
    from helpers import sp_weights
    return sp_weights(oracle_mod, N)
