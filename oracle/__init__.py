"""Python access to the plain C oracle (``ssd_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the
CPU-baseline leg of the benchmark, never by the library.  ``build()`` compiles
the C file with gcc into ``oracle/_build/libssd_oracle.so`` (FP64, the
oracle proper) and, with ``real="long"``, into ``libssd_oracle_ld.so``: the
same source with every value and operation in C ``long double`` (64-bit
significand on x86-64, IEEE binary128 on AArch64), an extended-precision
reference for measuring the round-off of FP64 evaluations.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ssd_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIBS = {"double": os.path.join(_OUT_DIR, "libssd_oracle.so"),
         "long": os.path.join(_OUT_DIR, "libssd_oracle_ld.so")}
_LIB_PATH = _LIBS["double"]
_DTYPE = {"double": np.float64, "long": np.longdouble}
_CREAL = {"double": ctypes.c_double, "long": ctypes.c_longdouble}
_loaded = {}

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False, real: str = "double") -> str:
    """Compile the oracle (plain C, no vectorisation flags, no FMA contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    path = _LIBS[real]
    if force or not os.path.exists(path) or os.path.getmtime(path) < os.path.getmtime(_SRC):
        tmp = path + f".tmp{os.getpid()}"
        extra = ["-DOR_REAL_LONG"] if real == "long" else []
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared", *extra, _SRC,
                               "-o", tmp, "-lm"])
        os.replace(tmp, path)
    return path


def lib(real: str = "double"):
    if real not in _loaded:
        build(real=real)
        L = ctypes.CDLL(_LIBS[real])
        R = _CREAL[real]
        rp = ctypes.POINTER(R)
        L.or_create.restype = ctypes.c_void_p
        L.or_create.argtypes = [ctypes.c_int, rp, ctypes.c_int, _ip, _ip, _ip, _ip, ctypes.c_int, _ip, ctypes.c_int,
                                _ip, ctypes.c_int, _ip, ctypes.c_int, _ip, R, R, R, ctypes.c_int, rp, ctypes.c_int,
                                rp, _ip, _ip, _ip, ctypes.c_char_p, ctypes.c_int]
        L.or_destroy.argtypes = [ctypes.c_void_p]
        L.or_residual.argtypes = [ctypes.c_void_p, rp, R, rp]
        L.or_residual_ex.argtypes = [ctypes.c_void_p, rp, R, rp, rp]
        L.or_step.argtypes = [ctypes.c_void_p, rp, rp, R, ctypes.c_int]
        L.or_step_rk54.argtypes = [ctypes.c_void_p, rp, rp, R, ctypes.c_int]
        L.or_rk54_tableau.argtypes = [rp, rp, rp]
        L.or_sp_coords.argtypes = [ctypes.c_void_p, R, rp]
        L.or_sp_jacobian.argtypes = [ctypes.c_void_p, rp]
        L.or_points.argtypes = [ctypes.c_int, rp, rp]
        L.or_gauss_legendre.argtypes = [ctypes.c_int, rp, rp]
        L.or_lagrange.argtypes = [rp, ctypes.c_int, rp, ctypes.c_int, rp, rp]
        L.or_projection.argtypes = [ctypes.c_int, R, R, rp, rp]
        L.or_rusanov.argtypes = [R, rp, rp, R, R, R, rp]
        L.or_face_info.restype = ctypes.c_char_p
        L.or_face_info.argtypes = [ctypes.c_void_p, _ip, _ip, _ip]
        L.or_mortar_list.restype = ctypes.c_int
        L.or_mortar_list.argtypes = [ctypes.c_void_p, R, _ip, _ip, rp, rp, rp, rp]
        L.or_mortar_list_zone.restype = ctypes.c_int
        L.or_mortar_list_zone.argtypes = [ctypes.c_void_p, ctypes.c_int, R, _ip, _ip, rp, rp, rp, rp]
        _loaded[real] = L
    return _loaded[real]


def _d(a):
    return a.ctypes.data_as(_dp)


def _r(a, real):
    """Pointer to a contiguous array of the oracle build's real type."""
    return a.ctypes.data_as(ctypes.POINTER(_CREAL[real]))


def _i(a):
    return a.ctypes.data_as(_ip)


def points(N: int):
    Xs, Xf = np.zeros(N), np.zeros(N + 1)
    lib().or_points(N, _d(Xs), _d(Xf))
    return Xs, Xf


def gauss_legendre(n: int):
    x, w = np.zeros(n), np.zeros(n)
    lib().or_gauss_legendre(n, _d(x), _d(w))
    return x, w


def lagrange(nodes, x):
    nodes = np.ascontiguousarray(nodes, dtype=np.float64)
    x = np.ascontiguousarray(np.atleast_1d(x), dtype=np.float64)
    val = np.zeros((len(x), len(nodes)))
    der = np.zeros((len(x), len(nodes)))
    lib().or_lagrange(_d(nodes), len(nodes), _d(x), len(x), _d(val), _d(der))
    return val, der


def projection(N: int, o: float, s: float):
    Pf, Pb = np.zeros((N, N)), np.zeros((N, N))
    lib().or_projection(N, o, s, _d(Pf), _d(Pb))
    return Pf, Pb


def rusanov(gamma, qL, qR, n, vgn=0.0):
    """Rusanov common normal flux of the oracle (Sec. 3.1) for conservative
    states qL, qR, unit normal n from L to R and normal grid velocity vgn."""
    qL = np.ascontiguousarray(qL, dtype=np.float64)
    qR = np.ascontiguousarray(qR, dtype=np.float64)
    out = np.zeros(4)
    lib().or_rusanov(float(gamma), _d(qL), _d(qR), float(n[0]), float(n[1]), float(vgn), _d(out))
    return out


def rk54_tableau():
    A, b, c = np.zeros((5, 5)), np.zeros(5), np.zeros(5)
    lib().or_rk54_tableau(_d(A), _d(b), _d(c))
    return A, b, c


def params_array(params) -> np.ndarray:
    return np.array([params.gamma, params.Rgas, params.mu, params.prandtl, params.omega,
                     float(params.viscous), params.T_wall, params.rho_inf, params.u_inf, params.v_inf,
                     params.p_inf], dtype=np.float64)


class Oracle:
    """One mesh + order + flow parameters; residual and SSP-RK3 steps.

    real="double": the FP64 oracle (results are float64 arrays); real="long":
    the extended-precision build (inputs converted exactly, results returned
    as numpy.longdouble arrays)."""

    def __init__(self, mesh: dict, N: int, params, real: str = "double"):
        L = lib(real)
        self.real = real
        self._dt = _DTYPE[real]
        self.params = params
        self._ext = None
        self.N = N
        self.mesh = mesh
        self.E = int(len(mesh["elem_nodes"]))
        self._keep = []

        def arr(x, dt):
            a = np.ascontiguousarray(x, dtype=dt)
            self._keep.append(a)
            return a

        xy = arr(mesh["xy"], self._dt)
        en = arr(mesh["elem_nodes"], np.int32)
        zone = arr(mesh["elem_zone"], np.int32)
        arc = arr(mesh["edge_arc"], np.int32)
        enode = arr(mesh["edge_nodes"], np.int32) if "edge_nodes" in mesh else None
        bf = arr(mesh["bfaces"], np.int32)
        pf = arr(mesh["pfaces"], np.int32)
        Lf = arr(mesh["ifaces_L"], np.int32)
        Rf = arr(mesh["ifaces_R"], np.int32)
        prm = arr(params_array(params), self._dt)
        # further rotating zones 2, 3, ...: centre, radius, angular velocity, interface lists
        extra = mesh.get("zones", [])
        xz = arr(np.array([[z["center"][0], z["center"][1], z["r_interface"], z["omega"]] for z in extra],
                          dtype=np.float64).reshape(-1, 4), self._dt)
        xcnt = arr(np.array([[len(z["ifaces_L"]), len(z["ifaces_R"])] for z in extra],
                            dtype=np.int32).reshape(-1, 2), np.int32)
        xfaces = arr(np.concatenate([np.asarray(z[k], dtype=np.int32).reshape(-1, 2) for z in extra
                                     for k in ("ifaces_L", "ifaces_R")] + [np.zeros((1, 2), np.int32)]),
                     np.int32)
        azone = arr(mesh["elem_arc_zone"], np.int32) if "elem_arc_zone" in mesh else None
        err = ctypes.create_string_buffer(256)
        rl = self.real
        self._h = L.or_create(len(xy), _r(xy, rl), self.E, _i(en), _i(zone), _i(arc),
                              _i(enode) if enode is not None else None, len(bf), _i(bf), len(pf),
                              _i(pf), len(Lf), _i(Lf), len(Rf), _i(Rf), float(mesh["center"][0]),
                              float(mesh["center"][1]), float(mesh["r_interface"]), N, _r(prm, rl), len(extra),
                              _r(xz, rl), _i(xcnt), _i(xfaces), _i(azone) if azone is not None else None, err, 256)
        if not self._h:
            raise ValueError("oracle mesh set-up failed: " + err.value.decode())

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib(self.real).or_destroy(h)
            self._h = None

    @property
    def shape(self):
        return (self.E, 4, self.N, self.N)

    def extended(self):
        """The same mesh, order and parameters in the extended-precision build
        (created once, on first use)."""
        if self.real == "long":
            return self
        if self._ext is None:
            self._ext = Oracle(self.mesh, self.N, self.params, real="long")
        return self._ext

    def sp_coords(self, t: float = 0.0):
        out = np.zeros((self.E, self.N, self.N, 2), dtype=self._dt)
        lib(self.real).or_sp_coords(self._h, t, _r(out, self.real))
        return out[..., 0], out[..., 1]

    def sp_jacobian(self):
        out = np.zeros((self.E, self.N, self.N), dtype=self._dt)
        lib(self.real).or_sp_jacobian(self._h, _r(out, self.real))
        return out

    def residual(self, Q, t: float = 0.0):
        Q = np.ascontiguousarray(Q, dtype=self._dt).reshape(self.shape)
        R = np.zeros(self.shape, dtype=self._dt)
        lib(self.real).or_residual(self._h, _r(Q, self.real), t, _r(R, self.real))
        return R

    def residual_with_scale(self, Q, t: float = 0.0):
        """Residual and, per point, the summed magnitude of its divergence terms."""
        Q = np.ascontiguousarray(Q, dtype=self._dt).reshape(self.shape)
        R, S = np.zeros(self.shape, dtype=self._dt), np.zeros(self.shape, dtype=self._dt)
        lib(self.real).or_residual_ex(self._h, _r(Q, self.real), t, _r(R, self.real), _r(S, self.real))
        return R, S

    def step(self, Q, t: float, dt: float, nsteps: int = 1, rk_stages: int = 3):
        """rk_stages 3: SSP-RK3 (Shu-Osher); 5: the five-stage fourth-order SSP-RK."""
        Q = np.array(Q, dtype=self._dt, order="C").reshape(self.shape)
        tt = np.array([t], dtype=self._dt)
        L = lib(self.real)
        fn = L.or_step_rk54 if rk_stages == 5 else L.or_step
        fn(self._h, _r(Q, self.real), _r(tt, self.real), dt, nsteps)
        return Q, float(tt[0])

    def face_info(self):
        n = 4 * self.E
        kind, nbr, rev = np.zeros(n, np.int32), np.zeros(n, np.int32), np.zeros(n, np.int32)
        lib(self.real).or_face_info(self._h, _i(kind), _i(nbr), _i(rev))
        return kind, nbr, rev

    def mortars(self, t: float, zone: int = 1):
        """Mortars of rotating zone ``zone``'s interface at time t (lf / rf index
        that interface's sorted L / R lists)."""
        z = self.mesh if zone == 1 else self.mesh["zones"][zone - 2]
        n = len(z["ifaces_L"]) + len(z["ifaces_R"])
        lf, rf = np.zeros(max(n, 1), np.int32), np.zeros(max(n, 1), np.int32)
        oL, sL, oR, sR = (np.zeros(max(n, 1), dtype=self._dt) for _ in range(4))
        rl = self.real
        k = lib(rl).or_mortar_list_zone(self._h, zone, t, _i(lf), _i(rf), _r(oL, rl), _r(sL, rl), _r(oR, rl),
                                        _r(sR, rl))
        return {"lf": lf[:k], "rf": rf[:k], "oL": oL[:k], "sL": sL[:k], "oR": oR[:k], "sR": sR[:k]}

    def state_from(self, field_fn, t: float = 0.0):
        """Sample an analytic field at the SPs -> Q array [E][4][N][N]."""
        x, y = self.sp_coords(t)
        q = field_fn(x, y)  # (..., 4)
        return np.ascontiguousarray(np.moveaxis(q, -1, 1))
