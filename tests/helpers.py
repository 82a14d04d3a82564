"""Shared test helpers: quadrature weights of the SP rule, small meshes."""
import math

import numpy as np

from ssd_inputs import meshes


def sp_weights(oracle_mod, N):
    """w_i = int_0^1 h_i(x) dx, computed with numpy's Gauss-Legendre rule."""
    Xs, _ = oracle_mod.points(N)
    z, w = np.polynomial.legendre.leggauss(N + 4)
    val, _ = oracle_mod.lagrange(Xs, 0.5 * (1 + z))
    return (0.5 * w[:, None] * val).sum(axis=0)


def small_rotor(scale=1, shift_L=0.0, shift_R=0.0, n_hole=6, n_core=4):
    return meshes.rotor_mesh(half_width=10.0, n_cart=16 * scale, n_hole=n_hole * scale, r_interface=3.0,
                             n_core=n_core * scale, core_half=1.5, n_ring_in=3 * scale,
                             n_ring_out=2 * scale, shift_L=shift_L, shift_R=shift_R)


def small_twin(omega2=-0.45, n_core2=None, shift_L=0.0, shift_R=0.0):
    """Two rotating disks in a periodic 12 x 6 box (384 cells)."""
    return meshes.twin_rotor_mesh(half_width=3.0, n_cart=12, n_hole=8, r_interface=1.5, n_core=4,
                                  core_half=0.6, n_ring_in=2, n_ring_out=2, omega2=omega2,
                                  shift_L=shift_L, shift_R=shift_R, n_core2=n_core2)


def small_row(n_rotors, omegas, shift_L=0.0, n_cores=None):
    """A row of n_rotors small disks (zones 1 .. n_rotors)."""
    return meshes.rotor_row_mesh(n_rotors, half_width=3.0, n_cart=12, n_hole=8, r_interface=1.5, n_core=4,
                                 core_half=0.6, n_ring_in=2, n_ring_out=2, omegas=omegas, shift_L=shift_L,
                                 n_cores=n_cores)


def face_kinds(mesh):
    """Per element: True if the cell has a curved edge or a non-conforming face."""
    E = len(mesh["elem_nodes"])
    special = mesh["edge_arc"].sum(axis=1) > 0
    for key in ("ifaces_L", "ifaces_R"):
        for e, f in mesh[key]:
            special[e] = True
    for row in mesh["pfaces"]:
        special[row[0]] = special[row[2]] = True
    for row in mesh["bfaces"]:
        special[row[0]] = True
    return special


def neighbours_of(mesh, mask):
    """Elements sharing a node with an element in mask."""
    en = mesh["elem_nodes"]
    bad_nodes = np.zeros(len(mesh["xy"]), dtype=bool)
    bad_nodes[en[mask].ravel()] = True
    return bad_nodes[en].any(axis=1)


def rel_err(a, b):
    """max |a-b| / max|b| per conservative variable (axis 1)."""
    num = np.abs(a - b).max(axis=(0, 2, 3))
    den = np.abs(b).max(axis=(0, 2, 3))
    return num / den


def random_cell_states(E, seed, gamma=1.4):
    """A seeded random constant state per cell, [E][4] conservative (rho, p
    in [0.5, 1.5], u, v in [-0.5, 0.5]): O(1) jumps on every face."""
    rng = np.random.Generator(np.random.PCG64(seed))
    rho, u, v, p = (rng.uniform(0.5, 1.5, E), rng.uniform(-0.5, 0.5, E), rng.uniform(-0.5, 0.5, E),
                    rng.uniform(0.5, 1.5, E))
    return np.stack([rho, rho * u, rho * v, p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)], axis=1)


def piecewise_constant(Qc, N):
    """[E][4][N][N] state holding Qc[e] at every solution point of cell e."""
    E = len(Qc)
    return np.ascontiguousarray(np.broadcast_to(np.asarray(Qc)[:, :, None, None], (E, 4, N, N)))
