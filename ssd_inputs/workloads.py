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
    rk_stages: int = 3
    # free stream: the inlet state and the outlet pressure
    rho_inf: float = 1.0
    u_inf: float = 0.0
    v_inf: float = 0.0
    p_inf: float = 1.0


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


def vortex_family(N=4, scale=1):
    """The vortex configuration's mesh refined ``scale`` times (h / scale),
    its flow parameters and a stable step: (mesh, FlowParams, dt)."""
    return _vortex(N, scale)


def _vortex(N=4, scale=1):
    mesh = meshes.rotor_mesh(half_width=10.0, n_cart=int(round(64 * scale)), n_hole=int(round(24 * scale)),
                             r_interface=3.0, n_core=int(round(24 * scale)), core_half=1.5,
                             n_ring_in=int(round(16 * scale)), n_ring_out=max(1, int(round(4 * scale))))
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


def _twin_rotor(N=6):
    # [-20,20] x [-10,10], h = 0.08, two disks r = 2 about (-10, 0) and (10, 0)
    # turning in opposite senses: 123,450 quads
    mesh = meshes.twin_rotor_mesh(half_width=10.0, n_cart=250, n_hole=60, r_interface=2.0, n_core=25,
                                  core_half=1.0, n_ring_in=10, n_ring_out=5, omega2=-0.5)
    prm = FlowParams(gamma=1.4, Rgas=1.0, omega=0.5, viscous=0)
    h = 0.04
    dt = 0.1 * h / ((1.0 + math.sqrt(1.4) + 2.0) * N * N)
    return mesh, prm, dt


def ellipse_params(omega=0.3, mach=0.2, re=1000.0):
    """Free stream rho = U = T = 1 along +x at Mach M: p_inf = R = 1/(gamma M^2);
    mu from Re on the major axis (length 1); isothermal body at T = 1."""
    gamma = 1.4
    p_inf = 1.0 / (gamma * mach * mach)
    return FlowParams(gamma=gamma, Rgas=p_inf, mu=1.0 / re, prandtl=0.72, omega=omega, viscous=1, T_wall=1.0,
                      rho_inf=1.0, u_inf=1.0, v_inf=0.0, p_inf=p_inf)


def _ellipse(N=5, scale=1.0, omega=0.3, **mesh_kw):
    if scale != 1.0:
        mesh_kw.setdefault("n_theta", max(16, 4 * int(round(32 * scale))))
        mesh_kw.setdefault("n_inner", max(3, int(round(40 * scale))))
        mesh_kw.setdefault("n_outer", max(4, int(round(117 * scale))))
    mesh = meshes.ellipse_mesh(**mesh_kw)
    prm = ellipse_params(omega=omega)
    c = math.sqrt(prm.gamma * prm.p_inf / prm.rho_inf)
    dt = stable_dt(mesh, N, prm, 1.0 + c + 2.0 * omega)
    return mesh, prm, dt


def tank_params(omega=1.0, mach=0.1, re=100.0, r_hub=0.5):
    """Stirred tank: velocity scale = hub wall speed U = omega r_hub at Mach M
    (R = (U/M)^2 / (gamma T) with T = 1), Re on the hub diameter 2 r_hub,
    isothermal walls at T = 1; the tank starts at rest."""
    gamma = 1.4
    U = omega * r_hub
    c = U / mach
    return FlowParams(gamma=gamma, Rgas=c * c / gamma, mu=U * 2.0 * r_hub / re, prandtl=0.72, omega=omega,
                      viscous=1, T_wall=1.0)


def _tank(N=4, **mesh_kw):
    mesh = meshes.stirred_tank_mesh(**mesh_kw)
    prm = tank_params()
    c = math.sqrt(prm.gamma * prm.Rgas)
    # the paper's step is 1e-4; the explicit limit of this mesh at this N is smaller
    dt = min(1e-4, stable_dt(mesh, N, prm, c + prm.omega * 3.0))
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
    if name == "ellipse_n5":
        mesh, prm, dt = _ellipse(5)
        return Workload(name, "Navier-Stokes flow past a rotating ellipse (axes 1:0.2), Re=1000, Mach 0.2, "
                        "rotating disk r<=2 at omega=0.3, 20096 curvilinear quads (12-node cubic cells "
                        "around the body), N=5 (p=4)", mesh, 5, prm, dt, 10000)
    if name == "tank_n4":
        mesh, prm, dt = _tank(4)
        return Workload(name, "2D stirred tank: rotating hub r=0.5 with 6 adiabatic blades (r 1-2, "
                        "thickness 0.1), sliding interface r=3, isothermal tank wall r=5 with 4 baffles "
                        "(height 1, thickness 0.1); omega=1, Re=100, Mach 0.1 at the hub; 14752 quads, "
                        "N=4 (p=3)", mesh, 4, prm, dt, 1000)
    if name == "rotor_n6":
        mesh, prm, dt = _rotor_large(6)
        return Workload(name, "vortex through rotor: periodic [-20,20]^2, rotating disk r<=4, "
                        "about 247k quads, N=6 (p=5), Euler", mesh, 6, prm, dt, 100)
    if name == "twin_rotor_n6":
        mesh, prm, dt = _twin_rotor(6)
        return Workload(name, "vortex between two counter-rotating rotors (two rotating zones, two "
                        "sliding interfaces): periodic [-20,20]x[-10,10], disks r<=2 about (-10,0) at "
                        "omega=0.5 and (10,0) at omega=-0.5, 123,450 quads, N=6 (p=5), Euler", mesh, 6,
                        prm, dt, 100)
    raise KeyError(name)


WORKLOADS = ("couette_n3", "vortex_n4", "vortex_n5", "ellipse_n5", "tank_n4", "rotor_n6", "twin_rotor_n6")


def min_edge(mesh) -> float:
    import numpy as np
    xy, en = mesh["xy"], mesh["elem_nodes"]
    d = [np.linalg.norm(xy[en[:, a]] - xy[en[:, b]], axis=1) for a, b in ((0, 1), (1, 2), (2, 3), (3, 0))]
    return float(np.min(d))


def stable_dt(mesh, N, prm, speed, cfl=0.1):
    """Explicit step from the smallest edge: acoustic/convective limit
    h / (speed N^2), and for viscous flow the diffusive limit h^2 / (nu N^4)."""
    h = min_edge(mesh)
    dt = cfl * h / (speed * N * N)
    if prm.viscous and prm.mu > 0:
        dt = min(dt, 0.25 * cfl * h * h / (prm.mu * N ** 4))
    return dt


def batch_cases(n=64, seed=1503, min_cells=1000, max_cells=8000):
    """Seeded mix of independent cases for the batched form, drawn uniformly
    from three families: Couette (viscous, walls), rotor (Euler vortex
    through a rotating disk) and rotating ellipse (viscous, slip / inlet /
    outlet, cubic cells); log-uniform cell counts, p in {2,..,5}, omega in
    U[0.1, 1].  Returns a list of (name, mesh, p, FlowParams, dt)."""
    import numpy as np
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for k in range(n):
        target = math.exp(rng.uniform(math.log(min_cells), math.log(max_cells)))
        p = int(rng.integers(2, 6))
        omega = float(rng.uniform(0.1, 1.0))
        N = p + 1
        family = rng.uniform()
        if family >= 2.0 / 3.0:
            # ellipse family: about 20096 s^2 cells
            mesh, prm, dt = _ellipse(N, scale=math.sqrt(target / 20096.0), omega=omega)
            out.append((f"ellipse{k}", mesh, p, prm, dt))
        elif family >= 1.0 / 3.0:
            # rotor family: about 6016 s^2 cells
            s = math.sqrt(target / 6016.0)
            nh = max(4, 2 * int(round(12 * s)))
            nc = max(nh + 6, 2 * int(round(32 * s)))
            if (nc - nh) % 2:
                nc += 1
            mesh = meshes.rotor_mesh(half_width=10.0, n_cart=nc, n_hole=nh, r_interface=3.0,
                                     n_core=max(2, int(round(24 * s))), core_half=1.5,
                                     n_ring_in=max(2, int(round(16 * s))),
                                     n_ring_out=max(2, int(round(4 * s))))
            prm = FlowParams(gamma=1.4, Rgas=1.0, omega=omega, viscous=0)
            dt = stable_dt(mesh, N, prm, 2.0 + math.sqrt(1.4) + 3.0 * omega)
            out.append((f"rotor{k}", mesh, p, prm, dt))
        else:
            # Couette family: nr x 8m rotating + nr x 10m stationary cells
            nr = max(2, int(round(math.sqrt(target / 72.0))))
            mm = max(1, int(round(target / (18.0 * nr))))
            mesh = meshes.couette_mesh(nr, 8 * mm, nr, 10 * mm)
            U = omega
            c = U / 0.1
            prm = FlowParams(gamma=1.4, Rgas=c * c / 1.4, mu=U / 10.0, prandtl=0.72, omega=omega, viscous=1,
                             T_wall=1.0)
            dt = stable_dt(mesh, N, prm, c + U)
            out.append((f"couette{k}", mesh, p, prm, dt))
    return out
