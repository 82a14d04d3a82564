"""Synthetic quadrilateral meshes for the sliding-mesh SD workloads.

The paper's meshes exist only as figures, so these generators build meshes of
the same kind: a rotating inner zone and a stationary outer zone that meet on
a circular sliding interface (Sec. 3.2), conforming quads inside each zone,
periodic or wall boundaries outside.  They hold no part of the SD method: they
only place nodes and list cells, boundary faces, periodic face pairs and the
two sides of the interface.

Mesh format (a dict of numpy arrays; the same dict feeds the oracle and the
CUDA library):

``xy``          float64 (n_nodes, 2)  node coordinates
``elem_nodes``  int32 (E, 4)          corners n0..n3, counter-clockwise
``elem_zone``   int32 (E,)            0 stationary, z >= 1 rotating zone z
``edge_arc``    int32 (E, 4)          edge kind of local face f: 0 straight,
                                      1 circular arc about the centre of the
                                      cell's arc zone, 2 cubic
                                      through the corners and two edge nodes
``edge_nodes``  int32 (E, 4, 2)       (only when some edge is cubic) nodes at
                                      face parameter 1/3 and 2/3 of each cubic
                                      edge, -1 elsewhere
``bfaces``      int32 (nb, 3)         (elem, local face, bc tag)
``pfaces``      int32 (np, 4)         periodic pairs (eA, fA, eB, fB)
``ifaces_L``    int32 (nL, 2)         interface faces of the rotating zone
``ifaces_R``    int32 (nR, 2)         interface faces of the stationary zone
``center``      float64 (2,)          rotation centre of zone 1 (the centre of its
                                      interface circle)
``r_interface`` float                 radius of zone 1's sliding interface
``zones``       list (optional)       rotating zones 2, 3, ...: dicts with
                                      ``center``, ``r_interface``, ``omega``
                                      (its angular velocity), ``ifaces_L``,
                                      ``ifaces_R`` as above for that zone's
                                      own interface with zone 0
``elem_arc_zone`` int32 (E,) (optional) zone whose centre the cell's arc
                                      edges are drawn about (default: the
                                      cell's own zone, zone 1 for stationary
                                      cells)

Local faces follow the reference square [0,1]^2 with n0=(0,0), n1=(1,0),
n2=(1,1), n3=(0,1): f0 is eta=0 (n0->n1), f1 is xi=1 (n1->n2), f2 is eta=1
(n3->n2), f3 is xi=0 (n0->n3).

Boundary tags: 1 isothermal no-slip wall (moving with its zone), 2 slip wall,
3 inlet (free stream imposed), 4 outlet (free-stream pressure imposed),
5 adiabatic no-slip wall (moving with its zone).

A cell whose edges are cubic is the paper's 12-node cubic cell (corners plus
two nodes per edge): the transfinite map through its four edges is the
12-node serendipity map.
"""
from __future__ import annotations

import math

import numpy as np

BC_WALL = 1
BC_SLIP = 2
BC_INLET = 3
BC_OUTLET = 4
BC_ADIABATIC = 5

EDGE_STRAIGHT, EDGE_ARC, EDGE_CUBIC = 0, 1, 2

# corner pairs of the four local faces, in the order of their face parameter
FACE_CORNERS = ((0, 1), (1, 2), (3, 2), (0, 3))


class _NodeTable:
    """Node list with de-duplication by rounded coordinate (one table per zone,
    so that the two sides of a sliding interface never share a node)."""

    def __init__(self, offset: int = 0):
        self.offset = offset
        self.xy: list[tuple[float, float]] = []
        self.key: dict[tuple[int, int], int] = {}

    def add(self, x: float, y: float) -> int:
        k = (int(round(x * 1e9)), int(round(y * 1e9)))
        idx = self.key.get(k)
        if idx is None:
            idx = self.offset + len(self.xy)
            self.key[k] = idx
            self.xy.append((float(x), float(y)))
        return idx


class _MeshBuilder:
    def __init__(self, center=(0.0, 0.0)):
        self.center = np.asarray(center, dtype=np.float64)
        self.zones: list[_NodeTable] = []
        self.cells: list[list[int]] = []
        self.zone_of: list[int] = []
        self.arcs: list[list[int]] = []
        self.enodes: list[list[list[int]]] = []

    def node_table(self) -> _NodeTable:
        off = sum(len(z.xy) for z in self.zones)
        t = _NodeTable(off)
        self.zones.append(t)
        return t

    def all_xy(self) -> np.ndarray:
        pts = [p for z in self.zones for p in z.xy]
        return np.asarray(pts, dtype=np.float64).reshape(-1, 2)

    def add_cell(self, xy_lookup, corners, zone, arc_edges=(), cubic_edges=None):
        """Add a quad given 4 node ids in either orientation.  ``arc_edges``
        lists unordered node-id pairs whose edge is a circular arc;
        ``cubic_edges`` maps an ordered corner pair (a, b) to the edge nodes
        at 1/3 and 2/3 of the way from a to b."""
        c = list(corners)
        p = np.array([xy_lookup(n) for n in c])
        area2 = 0.0
        for k in range(4):
            x0, y0 = p[k]
            x1, y1 = p[(k + 1) % 4]
            area2 += x0 * y1 - x1 * y0
        if area2 < 0:
            c = [c[0], c[3], c[2], c[1]]
        arcset = {frozenset(e) for e in arc_edges}
        arc = [1 if frozenset((c[a], c[b])) in arcset else 0 for a, b in FACE_CORNERS]
        en = [[-1, -1] for _ in range(4)]
        for f, (a, b) in enumerate(FACE_CORNERS):
            if not cubic_edges:
                break
            if (c[a], c[b]) in cubic_edges:
                m1, m2 = cubic_edges[(c[a], c[b])]
            elif (c[b], c[a]) in cubic_edges:
                m2, m1 = cubic_edges[(c[b], c[a])]
            else:
                continue
            arc[f] = EDGE_CUBIC
            en[f] = [int(m1), int(m2)]
        self.cells.append(c)
        self.zone_of.append(zone)
        self.arcs.append(arc)
        self.enodes.append(en)
        return len(self.cells) - 1


def _face_of(cell: list[int], a: int, b: int) -> int:
    for f, (i, j) in enumerate(FACE_CORNERS):
        if {cell[i], cell[j]} == {a, b}:
            return f
    raise ValueError("edge not in cell")


def _finish(mb: _MeshBuilder, bfaces, pfaces, ifL, ifR, r_interface, zones=None, arc_zone=None) -> dict:
    out = {
        "xy": mb.all_xy(),
        "elem_nodes": np.asarray(mb.cells, dtype=np.int32).reshape(-1, 4),
        "elem_zone": np.asarray(mb.zone_of, dtype=np.int32),
        "edge_arc": np.asarray(mb.arcs, dtype=np.int32).reshape(-1, 4),
        "bfaces": np.asarray(bfaces, dtype=np.int32).reshape(-1, 3),
        "pfaces": np.asarray(pfaces, dtype=np.int32).reshape(-1, 4),
        "ifaces_L": np.asarray(ifL, dtype=np.int32).reshape(-1, 2),
        "ifaces_R": np.asarray(ifR, dtype=np.int32).reshape(-1, 2),
        "center": mb.center.copy(),
        "r_interface": float(r_interface),
    }
    if any(k == EDGE_CUBIC for row in mb.arcs for k in row):
        out["edge_nodes"] = np.asarray(mb.enodes, dtype=np.int32).reshape(-1, 4, 2)
    if zones:
        out["zones"] = [{"center": np.asarray(z["center"], dtype=np.float64),
                         "r_interface": float(z["r_interface"]), "omega": float(z["omega"]),
                         "ifaces_L": np.asarray(z["ifaces_L"], dtype=np.int32).reshape(-1, 2),
                         "ifaces_R": np.asarray(z["ifaces_R"], dtype=np.int32).reshape(-1, 2)}
                        for z in zones]
    if arc_zone is not None:
        out["elem_arc_zone"] = np.asarray(arc_zone, dtype=np.int32)
    return out


def _ring(mb, table, zone, inner_pts, outer_pts, nlayers, inner_is_arc, outer_is_arc):
    """Structured ring between two closed point loops with equal point counts
    (counter-clockwise).  Layer l sits at blend lambda_l between them.
    Returns (cells, node ids of inner loop, node ids of outer loop)."""
    m = len(inner_pts)
    lam = np.linspace(0.0, 1.0, nlayers + 1)
    ids = np.zeros((nlayers + 1, m), dtype=np.int64)
    for l in range(nlayers + 1):
        for k in range(m):
            if l == 0:
                x, y = inner_pts[k]
            elif l == nlayers:
                x, y = outer_pts[k]
            else:
                x = (1 - lam[l]) * inner_pts[k][0] + lam[l] * outer_pts[k][0]
                y = (1 - lam[l]) * inner_pts[k][1] + lam[l] * outer_pts[k][1]
            ids[l, k] = table.add(x, y)
    look = _lookup(mb)
    cells = []
    for l in range(nlayers):
        for k in range(m):
            k1 = (k + 1) % m
            a, b, c, d = ids[l, k], ids[l + 1, k], ids[l + 1, k1], ids[l, k1]
            arcs = []
            if l == 0 and inner_is_arc:
                arcs.append((a, d))
            if l == nlayers - 1 and outer_is_arc:
                arcs.append((b, c))
            cells.append(mb.add_cell(look, [a, b, c, d], zone, arcs))
    return cells, ids[0], ids[nlayers]


def _lookup(mb):
    def f(n):
        for z in mb.zones:
            if z.offset <= n < z.offset + len(z.xy):
                return z.xy[n - z.offset]
        raise KeyError(n)
    return f


def _circle(center, r, m, phi0):
    return [(center[0] + r * math.cos(phi0 + 2 * math.pi * k / m),
             center[1] + r * math.sin(phi0 + 2 * math.pi * k / m)) for k in range(m)]


def _square_loop(center, s, m_side):
    """Counter-clockwise points on the square of half-width s, starting at the
    lower-left corner, m_side segments per side."""
    cx, cy = center
    pts = []
    for side in range(4):
        for k in range(m_side):
            t = k / m_side
            if side == 0:
                pts.append((cx - s + 2 * s * t, cy - s))
            elif side == 1:
                pts.append((cx + s, cy - s + 2 * s * t))
            elif side == 2:
                pts.append((cx + s - 2 * s * t, cy + s))
            else:
                pts.append((cx - s, cy + s - 2 * s * t))
    return pts


def _interface_faces(mb, cells, loop_ids):
    """(elem, local face) of the cells whose edge joins consecutive loop nodes."""
    out = []
    m = len(loop_ids)
    edge_to_cell = {}
    for e in cells:
        c = mb.cells[e]
        for f, (i, j) in enumerate(FACE_CORNERS):
            edge_to_cell[frozenset((c[i], c[j]))] = (e, f)
    for k in range(m):
        out.append(edge_to_cell[frozenset((int(loop_ids[k]), int(loop_ids[(k + 1) % m])))])
    return out


def couette_mesh(nr_in=4, nth_in=32, nr_out=4, nth_out=40, r_i=1.0, r_m=1.5, r_o=2.0,
                 phi_in=0.0, phi_out=0.0) -> dict:
    """Annulus r_i<=r<=r_o split at r_m: inner ring rotating (zone 1), outer
    ring stationary, isothermal walls at r_i and r_o (Sec. 4.2).  Every
    constant-radius edge is an exact arc, so all cells are annular sectors."""
    mb = _MeshBuilder((0.0, 0.0))
    c = (0.0, 0.0)
    tin = mb.node_table()
    cells_in, loop_i0, loop_i1 = _polar_ring(mb, tin, 1, c, np.linspace(r_i, r_m, nr_in + 1),
                                             nth_in, phi_in)
    tout = mb.node_table()
    cells_out, loop_o0, loop_o1 = _polar_ring(mb, tout, 0, c, np.linspace(r_m, r_o, nr_out + 1),
                                              nth_out, phi_out)
    bfaces = []
    for e, f in _interface_faces(mb, cells_in, loop_i0):
        bfaces.append((e, f, BC_WALL))
    for e, f in _interface_faces(mb, cells_out, loop_o1):
        bfaces.append((e, f, BC_WALL))
    ifL = _interface_faces(mb, cells_in, loop_i1)
    ifR = _interface_faces(mb, cells_out, loop_o0)
    return _finish(mb, bfaces, [], ifL, ifR, r_m)


def _polar_ring(mb, table, zone, center, radii, nth, phi0):
    nl = len(radii) - 1
    ids = np.zeros((nl + 1, nth), dtype=np.int64)
    for l in range(nl + 1):
        for k in range(nth):
            phi = phi0 + 2 * math.pi * k / nth
            ids[l, k] = table.add(center[0] + radii[l] * math.cos(phi),
                                  center[1] + radii[l] * math.sin(phi))
    look = _lookup(mb)
    cells = []
    for l in range(nl):
        for k in range(nth):
            k1 = (k + 1) % nth
            a, b, c, d = ids[l, k], ids[l + 1, k], ids[l + 1, k1], ids[l, k1]
            cells.append(mb.add_cell(look, [a, b, c, d], zone, [(a, d), (b, c)]))
    return cells, ids[0], ids[nl]


def _rotor_disk(mb, table, zone, c, core_half, n_core, r_interface, n_ring_in, phi):
    """Rotating disk about c: a core square of n_core x n_core straight cells
    and an O-ring of n_ring_in layers from the core square to the circle
    (4 n_core arcs starting at angle phi).  Returns (ring cells, circle nodes)."""
    look = _lookup(mb)
    core_ids = np.zeros((n_core + 1, n_core + 1), dtype=np.int64)
    for i in range(n_core + 1):
        for j in range(n_core + 1):
            core_ids[i, j] = table.add(c[0] - core_half + 2 * core_half * i / n_core,
                                       c[1] - core_half + 2 * core_half * j / n_core)
    for j in range(n_core):
        for i in range(n_core):
            mb.add_cell(look, [core_ids[i, j], core_ids[i + 1, j], core_ids[i + 1, j + 1],
                               core_ids[i, j + 1]], zone)
    sq = _square_loop(c, core_half, n_core)
    circ_in = _circle(c, r_interface, 4 * n_core, phi)
    cells_in, _, loopL = _ring(mb, table, zone, sq, circ_in, n_ring_in, False, True)
    return cells_in, loopL


def _hole_ring(mb, table, c, r_interface, m_out, half, n_hole, n_ring_out, phi):
    """Stationary O-ring of n_ring_out layers from the circle about c (m_out
    arcs starting at angle phi) out to the square hole of half-width ``half``.
    Returns (ring cells, circle nodes)."""
    circ_out = _circle(c, r_interface, m_out, phi)
    hole = _square_loop(c, half, n_hole)
    cells_out, loopR, _ = _ring(mb, table, 0, circ_out, hole, n_ring_out, True, False)
    return cells_out, loopR


def _cartesian_with_holes(mb, table, x0, y0, h, nx, ny, holes):
    """nx x ny Cartesian cells of spacing h from (x0, y0), periodic in x and y,
    without the cells (i, j) inside any hole (ilo, ihi, jlo, jhi).  Returns the
    periodic face pairs."""
    look = _lookup(mb)
    cart = np.zeros((nx + 1, ny + 1), dtype=np.int64)
    for i in range(nx + 1):
        for j in range(ny + 1):
            cart[i, j] = table.add(x0 + i * h, y0 + j * h)
    cart_cell = {}
    for j in range(ny):
        for i in range(nx):
            if any(ilo <= i < ihi and jlo <= j < jhi for ilo, ihi, jlo, jhi in holes):
                continue
            cart_cell[(i, j)] = mb.add_cell(look, [cart[i, j], cart[i + 1, j],
                                                   cart[i + 1, j + 1], cart[i, j + 1]], 0)
    pf = []
    for j in range(ny):
        a, bb = cart_cell[(0, j)], cart_cell[(nx - 1, j)]
        pf.append((a, _face_of(mb.cells[a], cart[0, j], cart[0, j + 1]),
                   bb, _face_of(mb.cells[bb], cart[nx, j], cart[nx, j + 1])))
    for i in range(nx):
        a, bb = cart_cell[(i, 0)], cart_cell[(i, ny - 1)]
        pf.append((a, _face_of(mb.cells[a], cart[i, 0], cart[i + 1, 0]),
                   bb, _face_of(mb.cells[bb], cart[i, ny], cart[i + 1, ny])))
    return pf


def rotor_mesh(half_width=10.0, n_cart=64, n_hole=24, r_interface=3.0, n_core=24,
               core_half=1.5, n_ring_in=16, n_ring_out=4, shift_L=0.0, shift_R=0.0) -> dict:
    """Periodic square [-w,w]^2 with a rotating disk r<=r_interface (Sec. 4.1).

    Rotating zone: a core square of n_core x n_core straight cells and an
    O-ring of n_ring_in layers from the core square to the circle (4*n_core
    interface faces).  Stationary zone: an O-ring of n_ring_out layers from
    the circle (4*n_hole interface faces) out to a square hole of half-width
    n_hole*h/2 cut from an n_cart x n_cart Cartesian grid of spacing
    h = 2w/n_cart, periodic in x and y.  Only the edges lying on the circle
    are arcs; every other edge is straight.  ``shift_L`` / ``shift_R`` turn the
    circle nodes of either side by a small angle (the corner nodes of the
    square loops stay put).
    """
    h = 2.0 * half_width / n_cart
    b = n_hole * h / 2.0
    if n_hole % 2 or (n_cart - n_hole) % 2:
        raise ValueError("n_hole and n_cart - n_hole must be even")
    if not (core_half * math.sqrt(2) < r_interface < b):
        raise ValueError("need core square inside the circle inside the hole")
    c = (0.0, 0.0)
    mb = _MeshBuilder(c)
    tin = mb.node_table()
    cells_in, loopL = _rotor_disk(mb, tin, 1, c, core_half, n_core, r_interface, n_ring_in,
                                  -0.75 * math.pi + shift_L)
    tout = mb.node_table()
    cells_out, loopR = _hole_ring(mb, tout, c, r_interface, 4 * n_hole, b, n_hole, n_ring_out,
                                  -0.75 * math.pi + shift_R)
    lo = (n_cart - n_hole) // 2
    pf = _cartesian_with_holes(mb, tout, -half_width, -half_width, h, n_cart, n_cart,
                               [(lo, lo + n_hole, lo, lo + n_hole)])
    ifL = _interface_faces(mb, cells_in, loopL)
    ifR = _interface_faces(mb, cells_out, loopR)
    return _finish(mb, [], pf, ifL, ifR, r_interface)


def rotor_row_mesh(n_rotors=2, half_width=10.0, n_cart=64, n_hole=24, r_interface=3.0, n_core=24,
                   core_half=1.5, n_ring_in=16, n_ring_out=4, omegas=(-math.pi / 4,),
                   shift_L=0.0, shift_R=0.0, n_cores=None) -> dict:
    """A row of rotating disks in one periodic box (several rotating zones,
    each with its own sliding interface; Sec. 3.2 applied per interface).

    The box [-n w, n w] x [-w, w] (n = n_rotors) is an n n_cart x n_cart
    Cartesian grid of spacing h = 2w/n_cart, periodic in x and y, with n
    square holes of n_hole x n_hole cells centred at (-n w + (2k + 1) w, 0).
    Each hole holds the disk and the stationary O-ring of ``rotor_mesh``:
    zone k + 1 about the k-th centre.  Zone 1's angular velocity is the flow
    parameter omega; zones 2 .. n turn at ``omegas``.  Disk k has
    4 n_cores[k] interface faces (default n_core for all).  The stationary
    ring cells about disk k draw their arcs about its centre
    (``elem_arc_zone`` = k + 1).
    """
    n = n_rotors
    cores = [n_core] * n if n_cores is None else list(n_cores)
    if len(omegas) != n - 1 or len(cores) != n:
        raise ValueError("need n_rotors - 1 angular velocities and n_rotors core sizes")
    h = 2.0 * half_width / n_cart
    b = n_hole * h / 2.0
    if n_hole % 2 or n_cart % 2 or (n_cart - n_hole) % 2:
        raise ValueError("n_cart, n_hole and n_cart - n_hole must be even")
    if not (core_half * math.sqrt(2) < r_interface < b):
        raise ValueError("need core square inside the circle inside the hole")
    centres = [(-n * half_width + (2 * k + 1) * half_width, 0.0) for k in range(n)]
    mb = _MeshBuilder(centres[0])
    disks = []
    for k in range(n):
        t = mb.node_table()
        disks.append(_rotor_disk(mb, t, k + 1, centres[k], core_half, cores[k], r_interface, n_ring_in,
                                 -0.75 * math.pi + shift_L))
    tout = mb.node_table()
    arc_zone = [z if z else 1 for z in mb.zone_of]
    rings = []
    for k in range(n):
        first = len(mb.cells)
        rings.append(_hole_ring(mb, tout, centres[k], r_interface, 4 * n_hole, b, n_hole, n_ring_out,
                                -0.75 * math.pi + shift_R))
        arc_zone += [k + 1] * (len(mb.cells) - first)
    lo = n_cart // 2 - n_hole // 2
    pf = _cartesian_with_holes(mb, tout, -n * half_width, -half_width, h, n * n_cart, n_cart,
                               [(lo + k * n_cart, lo + k * n_cart + n_hole, lo, lo + n_hole) for k in range(n)])
    arc_zone += [1] * (len(mb.cells) - len(arc_zone))
    faces = [(_interface_faces(mb, disks[k][0], disks[k][1]), _interface_faces(mb, rings[k][0], rings[k][1]))
             for k in range(n)]
    zones = [{"center": centres[k], "r_interface": r_interface, "omega": omegas[k - 1],
              "ifaces_L": faces[k][0], "ifaces_R": faces[k][1]} for k in range(1, n)]
    return _finish(mb, [], pf, faces[0][0], faces[0][1], r_interface, zones=zones, arc_zone=arc_zone)


def twin_rotor_mesh(half_width=10.0, n_cart=64, n_hole=24, r_interface=3.0, n_core=24,
                    core_half=1.5, n_ring_in=16, n_ring_out=4, omega2=-math.pi / 4,
                    shift_L=0.0, shift_R=0.0, n_core2=None) -> dict:
    """Two disks (``rotor_row_mesh`` with n_rotors = 2) about (-w, 0) and
    (w, 0); zone 2 turns at ``omega2`` and has 4 n_core2 interface faces
    (default n_core).  With n_core2 = n_core the mesh is symmetric under the
    half turn about the origin."""
    return rotor_row_mesh(2, half_width, n_cart, n_hole, r_interface, n_core, core_half, n_ring_in,
                          n_ring_out, (omega2,), shift_L, shift_R,
                          None if n_core2 is None else (n_core, n_core2))


def periodic_box_mesh(n=4, half_width=1.0, rotating=False) -> dict:
    """Plain periodic Cartesian box without an interface (small pin cases)."""
    mb = _MeshBuilder((0.0, 0.0))
    t = mb.node_table()
    look = _lookup(mb)
    h = 2 * half_width / n
    ids = np.zeros((n + 1, n + 1), dtype=np.int64)
    for i in range(n + 1):
        for j in range(n + 1):
            ids[i, j] = t.add(-half_width + i * h, -half_width + j * h)
    cell = {}
    for j in range(n):
        for i in range(n):
            cell[(i, j)] = mb.add_cell(look, [ids[i, j], ids[i + 1, j], ids[i + 1, j + 1],
                                              ids[i, j + 1]], 1 if rotating else 0)
    pf = []
    for j in range(n):
        a, bb = cell[(0, j)], cell[(n - 1, j)]
        pf.append((a, _face_of(mb.cells[a], ids[0, j], ids[0, j + 1]),
                   bb, _face_of(mb.cells[bb], ids[n, j], ids[n, j + 1])))
    for i in range(n):
        a, bb = cell[(i, 0)], cell[(i, n - 1)]
        pf.append((a, _face_of(mb.cells[a], ids[i, 0], ids[i + 1, 0]),
                   bb, _face_of(mb.cells[bb], ids[i, n], ids[i + 1, n])))
    return _finish(mb, [], pf, [], [], 0.0)


def perturb_nodes(mesh: dict, amplitude: float, seed: int = 1503) -> dict:
    """Seeded random displacement of nodes that lie on no arc and on no
    periodic or outer boundary (gives skewed straight-sided cells)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in mesh.items()}
    xy = out["xy"]
    fixed = np.zeros(len(xy), dtype=bool)
    en, arc = mesh["elem_nodes"], mesh["edge_arc"]
    for e in range(len(en)):
        for f, (i, j) in enumerate(FACE_CORNERS):
            if arc[e, f]:
                fixed[en[e, i]] = fixed[en[e, j]] = True
    if "edge_nodes" in mesh:
        enodes = mesh["edge_nodes"]
        fixed[enodes[enodes >= 0]] = True
    for row in mesh["bfaces"]:
        e, f = row[0], row[1]
        i, j = FACE_CORNERS[f]
        fixed[en[e, i]] = fixed[en[e, j]] = True
    for row in mesh["pfaces"]:
        for e, f in ((row[0], row[1]), (row[2], row[3])):
            i, j = FACE_CORNERS[f]
            fixed[en[e, i]] = fixed[en[e, j]] = True
    # displacement bounded by a fraction of the shortest incident edge
    hmin = np.full(len(xy), np.inf)
    for e in range(len(en)):
        for f, (i, j) in enumerate(FACE_CORNERS):
            d = np.linalg.norm(xy[en[e, i]] - xy[en[e, j]])
            hmin[en[e, i]] = min(hmin[en[e, i]], d)
            hmin[en[e, j]] = min(hmin[en[e, j]], d)
    disp = rng.uniform(-1.0, 1.0, size=xy.shape) * amplitude * hmin[:, None]
    disp[fixed] = 0.0
    out["xy"] = xy + disp
    return out


def mesh_stats(mesh: dict) -> dict:
    return {
        "elements": int(len(mesh["elem_nodes"])),
        "rotating": int((mesh["elem_zone"] > 0).sum()),
        "curved": int((mesh["edge_arc"].sum(axis=1) > 0).sum()),
        "interface_L": int(len(mesh["ifaces_L"])),
        "interface_R": int(len(mesh["ifaces_R"])),
        "periodic_pairs": int(len(mesh["pfaces"])),
        "boundary_faces": int(len(mesh["bfaces"])),
    }


def _geometric(n: int, ratio: float) -> np.ndarray:
    """n + 1 increasing values from 0 to 1 whose steps grow by ``ratio``."""
    if abs(ratio - 1.0) < 1e-12:
        return np.linspace(0.0, 1.0, n + 1)
    k = np.arange(n + 1, dtype=np.float64)
    return (ratio ** k - 1.0) / (ratio ** n - 1.0)


def ellipse_mesh(a=0.5, b=0.1, r_interface=2.0, n_theta=128, n_inner=40, n_outer=117,
                 box=(-10.0, 30.0, -10.0, 10.0), inner_ratio=1.08, outer_ratio=1.01,
                 shift_L=0.0) -> dict:
    """Flow past a rotating elliptic cylinder (Sec. 4: rotating disk inside a
    rectangular channel).

    Rotating zone: an O-grid of ``n_theta`` x ``n_inner`` cells between the
    ellipse x = a cos t, y = b sin t and the circle r = r_interface; its grid
    lines are the linear blends (1 - s) E(t) + s C(t), i.e. ellipses of
    semi-axes (1-s) a + s r, (1-s) b + s r, every one of them represented by
    cubic edges (12-node cells); the layer spacing grows geometrically from
    the body.  Stationary zone: an O-grid of ``n_theta`` x ``n_outer`` cells
    from the circle to the rectangle ``box`` = (x0, x1, y0, y1); the corners
    of the rectangle are nodes, and the circle nodes of each side of the
    rectangle are spaced uniformly in angle within that side's angular range,
    so the two sides of the interface never match node for node.  Tags: the
    ellipse is an isothermal wall moving with the zone, x = x0 the inlet,
    x = x1 the outlet, y = y0 and y = y1 slip walls.
    """
    x0, x1, y0, y1 = box
    c = (0.0, 0.0)
    if not (max(a, b) < r_interface < min(-x0, x1, -y0, y1)):
        raise ValueError("need the ellipse inside the disk inside the box")
    mb = _MeshBuilder(c)
    # rotating zone ----------------------------------------------------------
    tin = mb.node_table()
    look = _lookup(mb)
    s_in = _geometric(n_inner, inner_ratio)

    def ring_pt(k, t):
        A = (1.0 - s_in[k]) * a + s_in[k] * r_interface
        B = (1.0 - s_in[k]) * b + s_in[k] * r_interface
        return A * math.cos(t), B * math.sin(t)

    dt = 2.0 * math.pi / n_theta
    ids = np.zeros((n_inner + 1, n_theta), dtype=np.int64)
    for k in range(n_inner + 1):
        for i in range(n_theta):
            ids[k, i] = tin.add(*ring_pt(k, shift_L + i * dt))
    cubic = {}
    for k in range(n_inner):
        for i in range(n_theta):
            t0 = shift_L + i * dt
            m1 = tin.add(*ring_pt(k, t0 + dt / 3.0))
            m2 = tin.add(*ring_pt(k, t0 + 2.0 * dt / 3.0))
            cubic[(int(ids[k, i]), int(ids[k, (i + 1) % n_theta]))] = (m1, m2)
    cells_in = []
    for k in range(n_inner):
        for i in range(n_theta):
            i1 = (i + 1) % n_theta
            p, q, r, s = ids[k, i], ids[k + 1, i], ids[k + 1, i1], ids[k, i1]
            arcs = [(q, r)] if k == n_inner - 1 else []
            cells_in.append(mb.add_cell(look, [p, q, r, s], 1, arcs, cubic))
    # stationary zone --------------------------------------------------------
    tout = mb.node_table()
    look = _lookup(mb)
    corners = [(x1, y0), (x1, y1), (x0, y1), (x0, y0)]  # counter-clockwise from lower right
    ang = [math.atan2(y, x) for x, y in corners]
    ang = [ang[0]] + [ang[0] + ((ang[j] - ang[0]) % (2 * math.pi)) for j in (1, 2, 3)] + [ang[0] + 2 * math.pi]
    span = [ang[j + 1] - ang[j] for j in range(4)]
    # nodes per rectangle side in proportion to its angular range (largest remainders)
    raw = [n_theta * sp / (2 * math.pi) for sp in span]
    cnt = [max(1, int(math.floor(v))) for v in raw]
    order = sorted(range(4), key=lambda j: raw[j] - math.floor(raw[j]), reverse=True)
    j = 0
    while sum(cnt) < n_theta:
        cnt[order[j % 4]] += 1
        j += 1
    while sum(cnt) > n_theta:
        jm = max(range(4), key=lambda q: cnt[q])
        cnt[jm] -= 1
    circ, rect, side_of = [], [], []
    for sd in range(4):
        pa, pb = corners[sd], corners[(sd + 1) % 4]
        for q in range(cnt[sd]):
            f = q / cnt[sd]
            t = ang[sd] + f * span[sd]
            circ.append((r_interface * math.cos(t), r_interface * math.sin(t)))
            rect.append((pa[0] + f * (pb[0] - pa[0]), pa[1] + f * (pb[1] - pa[1])))
            side_of.append(sd)
    s_out = _geometric(n_outer, outer_ratio)
    oid = np.zeros((n_outer + 1, n_theta), dtype=np.int64)
    for k in range(n_outer + 1):
        for i in range(n_theta):
            if k == 0:
                x, y = circ[i]
            elif k == n_outer:
                x, y = rect[i]
            else:
                x = (1 - s_out[k]) * circ[i][0] + s_out[k] * rect[i][0]
                y = (1 - s_out[k]) * circ[i][1] + s_out[k] * rect[i][1]
            oid[k, i] = tout.add(x, y)
    cells_out = []
    for k in range(n_outer):
        for i in range(n_theta):
            i1 = (i + 1) % n_theta
            p, q, r, s = oid[k, i], oid[k + 1, i], oid[k + 1, i1], oid[k, i1]
            arcs = [(p, s)] if k == 0 else []
            cells_out.append(mb.add_cell(look, [p, q, r, s], 0, arcs))
    # boundaries -------------------------------------------------------------
    bfaces = [(e, f, BC_WALL) for e, f in _interface_faces(mb, cells_in, ids[0])]
    side_tag = (BC_OUTLET, BC_SLIP, BC_INLET, BC_SLIP)
    for i, (e, f) in enumerate(_interface_faces(mb, cells_out, oid[n_outer])):
        bfaces.append((e, f, side_tag[side_of[i]]))
    ifL = _interface_faces(mb, cells_in, ids[n_inner])
    ifR = _interface_faces(mb, cells_out, oid[0])
    return _finish(mb, bfaces, [], ifL, ifR, r_interface)


def channel_mesh(nx=6, ny=4, lx=3.0, ly=2.0, tags=(BC_INLET, BC_OUTLET, BC_SLIP, BC_SLIP),
                 mapping=None, cubic=False, zone=0) -> dict:
    """Rectangle [0, lx] x [0, ly] of nx x ny cells (all in ``zone``; zone 1
    rotates about the origin) with boundary tags (left, right, bottom, top).  ``mapping`` (x, y) -> (X, Y) moves every
    node; with ``cubic`` each edge also gets the mapped points at 1/3 and 2/3
    of its length, i.e. the cells are 12-node cubic cells, and a mapping whose
    components are in the cubic serendipity span (x^a y^b with a + b <= 3, or
    x^3 y, x y^3) is then reproduced exactly by every cell."""
    mb = _MeshBuilder((0.0, 0.0))
    t = mb.node_table()
    look = _lookup(mb)
    fmap = mapping if mapping is not None else (lambda x, y: (x, y))
    hx, hy = lx / nx, ly / ny
    ids = np.zeros((nx + 1, ny + 1), dtype=np.int64)
    for i in range(nx + 1):
        for j in range(ny + 1):
            ids[i, j] = t.add(*fmap(i * hx, j * hy))
    cub = {}
    if cubic:
        for i in range(nx + 1):
            for j in range(ny + 1):
                if i < nx:  # edge (i, j) -> (i + 1, j)
                    cub[(int(ids[i, j]), int(ids[i + 1, j]))] = (
                        t.add(*fmap((i + 1.0 / 3.0) * hx, j * hy)), t.add(*fmap((i + 2.0 / 3.0) * hx, j * hy)))
                if j < ny:  # edge (i, j) -> (i, j + 1)
                    cub[(int(ids[i, j]), int(ids[i, j + 1]))] = (
                        t.add(*fmap(i * hx, (j + 1.0 / 3.0) * hy)), t.add(*fmap(i * hx, (j + 2.0 / 3.0) * hy)))
    cell = {}
    for j in range(ny):
        for i in range(nx):
            cell[(i, j)] = mb.add_cell(look, [ids[i, j], ids[i + 1, j], ids[i + 1, j + 1], ids[i, j + 1]], zone,
                                       (), cub)
    bf = []
    for j in range(ny):
        e = cell[(0, j)]
        bf.append((e, _face_of(mb.cells[e], ids[0, j], ids[0, j + 1]), tags[0]))
        e = cell[(nx - 1, j)]
        bf.append((e, _face_of(mb.cells[e], ids[nx, j], ids[nx, j + 1]), tags[1]))
    for i in range(nx):
        e = cell[(i, 0)]
        bf.append((e, _face_of(mb.cells[e], ids[i, 0], ids[i + 1, 0]), tags[2]))
        e = cell[(i, ny - 1)]
        bf.append((e, _face_of(mb.cells[e], ids[i, ny], ids[i + 1, ny]), tags[3]))
    return _finish(mb, bf, [], [], [], 0.0)


def _radii(segments):
    """Concatenate radial node lists: segments of (r0, r1, layers, ratio);
    ratio > 1 grows the spacing from r0, ratio < 1 shrinks it towards r1."""
    out = [segments[0][0]]
    for r0, r1, n, ratio in segments:
        if ratio >= 1.0:
            f = _geometric(n, ratio)
        else:
            f = 1.0 - _geometric(n, 1.0 / ratio)[::-1]
        out.extend(list(r0 + (r1 - r0) * f[1:]))
    return np.asarray(out)


def stirred_tank_mesh(r_hub=0.5, r_interface=3.0, r_tank=5.0, n_blades=6, blade_r=(1.0, 2.0), blade_t=0.1,
                      n_baffles=4, baffle_h=1.0, baffle_t=0.1, n_theta_in=168, n_theta_out=200,
                      layers_in=(10, 16, 14), layers_out=(20, 22), shift_L=0.0) -> dict:
    """Two-dimensional stirred tank (Sec. 4): a rotating hub wall r = r_hub with
    ``n_blades`` flat blades (radial extent ``blade_r``, thickness ``blade_t``),
    a sliding interface at r = r_interface, and a stationary tank wall r = r_tank
    carrying ``n_baffles`` flat baffles (height ``baffle_h``, thickness
    ``baffle_t``).  Polar grids in both zones (layers refined towards the hub
    and the tank wall); a blade or baffle removes the two cells on either side
    of its axis over its radial extent, and the grid lines that bound it are
    moved onto the plate's faces (offset +-t/2 from the axis), so blades and
    baffles are exact rectangles.  Tags: hub and tank wall and baffles
    isothermal walls moving with their zone, blades adiabatic walls."""
    c = (0.0, 0.0)
    if n_theta_in % n_blades or n_theta_out % n_baffles:
        raise ValueError("theta counts must be multiples of the blade / baffle counts")
    mb = _MeshBuilder(c)

    def zone_grid(table, zone, radii, n_theta, phi0, plates, lo, hi, on_circle_top):
        """plates: list of axis line indices; the plate spans layers lo..hi."""
        dth = 2.0 * math.pi / n_theta
        nl = len(radii) - 1
        axes = {j: phi0 + j * dth for j in plates}
        ids = np.zeros((nl + 1, n_theta), dtype=np.int64)
        for k in range(nl + 1):
            for j in range(n_theta):
                r, phi = radii[k], phi0 + j * dth
                x, y = r * math.cos(phi), r * math.sin(phi)
                for ja, th in axes.items():
                    side = (j - ja) % n_theta
                    if lo <= k <= hi and side in (1, n_theta - 1):
                        sgn = 1.0 if side == 1 else -1.0
                        h = 0.5 * (baffle_t if zone == 0 else blade_t)
                        along = math.sqrt(r * r - h * h) if (on_circle_top and k == nl) else r
                        x = along * math.cos(th) - sgn * h * math.sin(th)
                        y = along * math.sin(th) + sgn * h * math.cos(th)
                ids[k, j] = table.add(x, y)
        look = _lookup(mb)
        cells = []
        for k in range(nl):
            for j in range(n_theta):
                if lo <= k < hi and any((j - ja) % n_theta in (0, n_theta - 1) for ja in plates):
                    continue
                j1 = (j + 1) % n_theta
                p, q, r_, s = ids[k, j], ids[k + 1, j], ids[k + 1, j1], ids[k, j1]
                arcs = []
                if k == 0:
                    arcs.append((p, s))
                if k == nl - 1:
                    arcs.append((q, r_))
                cells.append(mb.add_cell(look, [p, q, r_, s], zone, arcs))
        return cells, ids

    def single_edges(cells):
        count = {}
        for e in cells:
            cl = mb.cells[e]
            for f, (i, j) in enumerate(FACE_CORNERS):
                count.setdefault(frozenset((cl[i], cl[j])), []).append((e, f))
        return {k: v[0] for k, v in count.items() if len(v) == 1}

    # rotating zone: hub .. blade root .. blade tip .. interface
    rin = _radii([(r_hub, blade_r[0], layers_in[0], 1.15), (blade_r[0], blade_r[1], layers_in[1], 1.0),
                  (blade_r[1], r_interface, layers_in[2], 1.0)])
    kb0, kb1 = layers_in[0], layers_in[0] + layers_in[1]
    tin = mb.node_table()
    blades = [b * (n_theta_in // n_blades) for b in range(n_blades)]
    cells_in, ids_in = zone_grid(tin, 1, rin, n_theta_in, shift_L, blades, kb0, kb1, False)
    # stationary zone: interface .. baffle root .. tank wall
    rout = _radii([(r_interface, r_tank - baffle_h, layers_out[0], 1.0),
                   (r_tank - baffle_h, r_tank, layers_out[1], 1.0 / 1.12)])
    tout = mb.node_table()
    baffles = [b * (n_theta_out // n_baffles) + n_theta_out // (2 * n_baffles) for b in range(n_baffles)]
    nlo = len(rout) - 1
    cells_out, ids_out = zone_grid(tout, 0, rout, n_theta_out, 0.0, baffles, layers_out[0], nlo, True)
    # boundaries: every unshared edge that is not on the interface
    ifL = _interface_faces(mb, cells_in, ids_in[-1])
    ifR = _interface_faces(mb, cells_out, ids_out[0])
    iface = set(map(tuple, ifL)) | set(map(tuple, ifR))
    bfaces = []
    hub = {int(n) for n in ids_in[0]}
    for edge, (e, f) in single_edges(cells_in).items():
        if (e, f) in iface:
            continue
        bfaces.append((e, f, BC_WALL if edge <= hub else BC_ADIABATIC))
    for edge, (e, f) in single_edges(cells_out).items():
        if (e, f) in iface:
            continue
        bfaces.append((e, f, BC_WALL))
    bfaces.sort()
    return _finish(mb, bfaces, [], ifL, ifR, r_interface)
