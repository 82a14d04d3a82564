"""Analytic flow fields used as initial states and exact solutions (Sec. 4).

Each function takes physical coordinates (and time) and returns the
conservative variables Q = [rho, rho u, rho v, E] (Sec. 2.1, Eq. Q) with
E = p/(gamma-1) + rho (u^2 + v^2)/2.  None of this is SD arithmetic: the
coordinates at which a field is sampled come from whichever side (oracle or
library) is being initialised.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate


def conservative(rho, u, v, p, gamma=1.4):
    rho = np.asarray(rho)
    u = np.broadcast_to(u, rho.shape)
    v = np.broadcast_to(v, rho.shape)
    p = np.broadcast_to(p, rho.shape)
    return np.stack([rho, rho * u, rho * v, p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)], axis=-1)


def uniform(x, y, rho=1.0, u=0.0, v=0.0, p=1.0, gamma=1.4):
    shape = np.shape(x)
    return conservative(np.full(shape, rho), u, v, np.full(shape, p), gamma)


def isentropic_vortex(x, y, t=0.0, eps=5.0 / (2.0 * math.pi), rc=1.0, u_inf=1.0, rho_inf=1.0,
                      p_inf=1.0, theta=0.0, x0=0.0, y0=0.0, gamma=1.4, period=None):
    """Euler vortex of Sec. 4.1 convected by a uniform mean flow.

    The Mach number entering the density/pressure dip is
    M = u_inf / sqrt(gamma p_inf / rho_inf), which is the value for which the
    printed formula is in radial equilibrium.  With the defaults
    (eps = 5/(2 pi), u_inf = rho_inf = p_inf = 1) this is the common
    strength-5 isentropic vortex.  ``period`` = (xmin, L) applies the
    periodic wrap of Eqs. xrnew/yrnew on a square of side L starting at xmin.
    """
    x = np.asarray(x)
    y = np.asarray(y)
    ubar, vbar = u_inf * math.cos(theta), u_inf * math.sin(theta)
    xr = x - x0 - ubar * t
    yr = y - y0 - vbar * t
    if period is not None:
        xmin, L = period
        # shift so that the domain starts at 0 before the floor formula
        xr = xr - np.floor((xr + x0 - xmin) / L) * L
        yr = yr - np.floor((yr + y0 - xmin) / L) * L
    mach = u_inf / math.sqrt(gamma * p_inf / rho_inf)
    r2 = xr * xr + yr * yr
    e1 = np.exp((1.0 - r2) / (2.0 * rc * rc))
    u = u_inf * (math.cos(theta) - eps * yr / rc * e1)
    v = u_inf * (math.sin(theta) + eps * xr / rc * e1)
    base = 1.0 - (gamma - 1.0) * (eps * mach) ** 2 / 2.0 * np.exp((1.0 - r2) / (rc * rc))
    rho = rho_inf * base ** (1.0 / (gamma - 1.0))
    p = p_inf * base ** (gamma / (gamma - 1.0))
    return conservative(rho, u, v, p, gamma)


def couette_velocity(r, omega_i=1.0, r_i=1.0, r_o=2.0):
    """Exact circumferential velocity of Sec. 4.2 (inner wall speed omega_i r_i,
    outer wall at rest)."""
    r = np.asarray(r, dtype=np.float64)
    return omega_i * r_i * (r_o / r - r / r_o) / (r_o / r_i - r_i / r_o)


class CouetteExact:
    """Steady compressible Taylor-Couette state with constant viscosity and
    isothermal walls at T_w.

    v_theta(r) is the incompressible profile (exact here too: the azimuthal
    momentum balance with constant mu does not involve rho).  The energy
    balance k (r T')'/r + mu (r d(v/r)/dr)^2 = 0 gives
    T = T_w + C1 ln r - mu b^2/(k r^2) + C2, with v = a r + b/r.  The radial
    balance dp/dr = rho v^2/r with p = rho R T is integrated numerically for
    rho, normalised so that rho(r_i) = rho_i.
    """

    def __init__(self, omega_i, r_i, r_o, mu, k, Rgas, T_w, rho_i=1.0, gamma=1.4):
        self.omega_i, self.r_i, self.r_o = omega_i, r_i, r_o
        self.mu, self.k, self.Rgas, self.T_w, self.gamma = mu, k, Rgas, T_w, gamma
        den = r_o / r_i - r_i / r_o
        self.a = -omega_i * r_i / r_o / den
        self.b = omega_i * r_i * r_o / den
        # T(r) = A + B ln r - mu b^2/(k r^2), T(r_i) = T(r_o) = T_w
        c = mu * self.b ** 2 / k
        M = np.array([[1.0, math.log(r_i)], [1.0, math.log(r_o)]])
        rhs = np.array([T_w + c / r_i ** 2, T_w + c / r_o ** 2])
        self.A, self.B = np.linalg.solve(M, rhs)
        self.rho_i = rho_i
        self._c = c

    def T(self, r):
        return self.A + self.B * np.log(r) - self._c / (np.asarray(r) ** 2)

    def v(self, r):
        return self.a * np.asarray(r) + self.b / np.asarray(r)

    def rho(self, r):
        r = np.atleast_1d(np.asarray(r, dtype=np.float64))
        out = np.empty_like(r)
        # d ln(rho T)/dr = v^2/(r R T)
        f = lambda s: self.v(s) ** 2 / (s * self.Rgas * self.T(s))
        for idx, rv in np.ndenumerate(r):
            val, _ = integrate.quad(f, self.r_i, rv, epsabs=1e-15, epsrel=1e-14, limit=200)
            out[idx] = self.rho_i * self.T(self.r_i) / self.T(rv) * math.exp(val)
        return out

    def state(self, x, y):
        x = np.asarray(x, dtype=np.float64)
        y = np.asarray(y, dtype=np.float64)
        r = np.sqrt(x * x + y * y)
        vt = self.v(r)
        rho = self.rho(r.ravel()).reshape(r.shape)
        T = self.T(r)
        p = rho * self.Rgas * T
        u = -vt * y / r
        v = vt * x / r
        return conservative(rho, u, v, p, self.gamma)


def random_smooth_state(x, y, seed=1503, amp=0.05, rho0=1.0, p0=1.0, u0=0.3, v0=-0.2, gamma=1.4,
                        kmax=2, scale=1.0):
    """Seeded smooth random state: a few random Fourier modes on top of a
    uniform flow (used for parity cases; positive density and pressure)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x = np.asarray(x, dtype=np.float64) / scale
    y = np.asarray(y, dtype=np.float64) / scale
    fields = []
    for _ in range(4):
        acc = np.zeros_like(x)
        for kx in range(-kmax, kmax + 1):
            for ky in range(-kmax, kmax + 1):
                a, ph = rng.uniform(-1, 1), rng.uniform(0, 2 * math.pi)
                acc += a * np.sin(kx * x + ky * y + ph)
        fields.append(acc / (2 * kmax + 1))
    rho = rho0 * (1 + amp * fields[0])
    u = u0 + amp * fields[1]
    v = v0 + amp * fields[2]
    p = p0 * (1 + amp * fields[3])
    return conservative(rho, u, v, p, gamma)


def noise(shape, seed=1503, amp=1e-3):
    rng = np.random.Generator(np.random.PCG64(seed))
    return amp * rng.standard_normal(shape)


def ellipse_start(x, y, rho_inf=1.0, u_inf=1.0, v_inf=0.0, p_inf=1.0, omega=0.0, a=0.5, b=0.1, width=1.0,
                  gamma=1.4):
    """Uniform density and pressure with a velocity that is the free stream far
    from the ellipse x^2/a^2 + y^2/b^2 = 1 and the body's rigid rotation
    omega x r on it: V = phi V_inf + (1 - phi) omega x r with
    phi = 1 - exp(-(s / width)^2), s = sqrt(x^2/a^2 + y^2/b^2) - 1.  A smooth
    start that already meets the no-slip condition (unlike the impulsively
    started free stream)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    s = np.sqrt((x / a) ** 2 + (y / b) ** 2) - 1.0
    phi = 1.0 - np.exp(-(np.maximum(s, 0.0) / width) ** 2)
    u = phi * u_inf - (1.0 - phi) * omega * y
    v = phi * v_inf + (1.0 - phi) * omega * x
    return conservative(np.full(x.shape, rho_inf), u, v, np.full(x.shape, p_inf), gamma)
