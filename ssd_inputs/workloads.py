"""Named workloads: mesh, polynomial order and flow parameters.

Non-dimensionalisation (the paper fixes gamma = 1.4 only): reference density
and temperature 1, R = 1/(gamma M^2) so that the reference speed is 1 at Mach
M; mu = rho U L / Re; Prandtl 0.72.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

from . import meshes


@dataclass
class FlowParams:
    gamma: float = 1.4
    Rgas: float = 1.0
    mu: float = 0.0
    prandtl: float = 0.72
    omega: float = 0.0
    viscous: int = 0
    T_wall: float = 1.0


@dataclass
class Workload:
    name: str
    description: str
    mesh: dict
    N: int
    params: FlowParams
    cfl_dt: float
    steps: int
    extra: dict = field(default_factory=dict)


def _couette(scale=1, N=3, omega=0.5, mach=0.1, re=10.0):
    # inner wall speed U = omega r_i is the velocity scale; Mach M_i = U / c
    mesh = meshes.couette_mesh(4 * scale, 32 * scale, 4 * scale, 40 * scale)
    U = omega * 1.0
    gamma = 1.4
    T_w = 1.0
    c = U / mach
    Rgas = c * c / (gamma * T_w)
    mu = 1.0 * U * 1.0 / re
    prm = FlowParams(gamma=gamma, Rgas=Rgas, mu=mu, prandtl=0.72, omega=omega, viscous=1,
                     T_wall=T_w)
    h = 0.5 / (4 * scale)
    dt = 0.1 * h / ((c + U) * N * N)
    return mesh, prm, dt


def _vortex(N=4, scale=1):
    mesh = meshes.rotor_mesh(half_width=10.0, n_cart=64 * scale, n_hole=24 * scale,
                             r_interface=3.0, n_core=24 * scale, core_half=1.5,
                             n_ring_in=16 * scale, n_ring_out=4 * scale)
    prm = FlowParams(gamma=1.4, Rgas=1.0, omega=math.pi / 4, viscous=0)
    h = 3.0 / 24 / scale
    dt = 0.1 * h / ((1.0 + math.sqrt(1.4) + 3.0 * math.pi / 4 * 0 + 2.0) * N * N)
    return mesh, prm, dt


def _rotor_large(N=6):
    # [-20,20]^2, h = 0.08, rotating disk r = 4: about 247k quads
    mesh = meshes.rotor_mesh(half_width=20.0, n_cart=500, n_hole=120, r_interface=4.0,
                             n_core=50, core_half=2.0, n_ring_in=20, n_ring_out=10)
    prm = FlowParams(gamma=1.4, Rgas=1.0, omega=0.5, viscous=0)
    h = 0.04
    dt = 0.1 * h / ((1.0 + math.sqrt(1.4) + 2.0) * N * N)
    return mesh, prm, dt


def build_workload(name: str) -> Workload:
    if name == "couette_n3":
        mesh, prm, dt = _couette()
        return Workload(name, "Taylor-Couette NS, annulus r in [1,2], inner ring 4x32 rotating "
                        "(omega=0.5), outer ring 4x40, N=3 (p=2), Mach 0.1, Re=10", mesh, 3, prm,
                        dt, 200)
    if name in ("vortex_n4", "vortex_n5"):
        N = int(name[-1])
        mesh, prm, dt = _vortex(N)
        return Workload(name, f"isentropic vortex (strength 5) on periodic [-10,10]^2, rotating "
                        f"disk r<=3 at omega=pi/4, N={N} (p={N-1}), Euler", mesh, N, prm, dt, 100)
    if name == "rotor_n6":
        mesh, prm, dt = _rotor_large(6)
        return Workload(name, "vortex through rotor: periodic [-20,20]^2, rotating disk r<=4, "
                        "about 247k quads, N=6 (p=5), Euler", mesh, 6, prm, dt, 100)
    raise KeyError(name)


WORKLOADS = ("couette_n3", "vortex_n4", "vortex_n5", "rotor_n6")
