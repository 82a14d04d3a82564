"""Thin Python binding of the C ABI in include/ssd.h (libssd.so).

Argument marshalling only: every step of the residual and of the time step
runs in the library's CUDA kernels.  Arrays may be numpy arrays (host memory)
or CUDA torch tensors (device memory; passed by data pointer).  The library
must have been built (``build()`` or ``__graft_entry__.build()``); importing
this module never falls back to anything else.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build_mod

_HERE = os.path.dirname(os.path.abspath(__file__))
# SSD_LIBRARY=debug selects the debug build (index checks in the kernels)
_DEBUG = os.environ.get("SSD_LIBRARY", "") == "debug"
LIB_PATH = os.path.join(_HERE, "_build", "libssd_debug.so" if _DEBUG else "libssd.so")

SD_OK = 0
SD_ERR_ARG = -1
SD_ERR_MESH = -2
SD_ERR_CUDA = -3
SD_ERR_NONPHYSICAL = -4
SD_ERR_TIMEOUT = -5
SD_ERR_UNSUPPORTED = -6
SD_PREC_FP64 = 0
SD_PREC_FP32 = 1
SD_PREC_FP32S = 2
SD_PREC_FP32_TF32 = 3

_c_int_p = ctypes.POINTER(ctypes.c_int)
_c_dbl_p = ctypes.POINTER(ctypes.c_double)


SD_MAX_ZONES = 4


class sd_zone(ctypes.Structure):
    _fields_ = [("center", ctypes.c_double * 2), ("r_interface", ctypes.c_double), ("omega", ctypes.c_double),
                ("n_iface_L", ctypes.c_int), ("iface_L", _c_int_p), ("n_iface_R", ctypes.c_int),
                ("iface_R", _c_int_p)]


class sd_mesh(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int), ("xy", _c_dbl_p), ("n_elems", ctypes.c_int),
                ("elem_nodes", _c_int_p), ("elem_zone", _c_int_p), ("edge_arc", _c_int_p),
                ("n_bfaces", ctypes.c_int), ("bfaces", _c_int_p), ("n_pfaces", ctypes.c_int),
                ("pfaces", _c_int_p), ("n_iface_L", ctypes.c_int), ("iface_L", _c_int_p),
                ("n_iface_R", ctypes.c_int), ("iface_R", _c_int_p), ("center", ctypes.c_double * 2),
                ("r_interface", ctypes.c_double), ("edge_nodes", _c_int_p), ("n_zones", ctypes.c_int),
                ("zones", ctypes.POINTER(sd_zone)), ("elem_arc_zone", _c_int_p)]


class sd_params(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("Rgas", ctypes.c_double), ("mu", ctypes.c_double),
                ("prandtl", ctypes.c_double), ("omega", ctypes.c_double), ("T_wall", ctypes.c_double),
                ("viscous", ctypes.c_int), ("precision", ctypes.c_int), ("stream", ctypes.c_void_p),
                ("rk_stages", ctypes.c_int), ("rho_inf", ctypes.c_double), ("u_inf", ctypes.c_double),
                ("v_inf", ctypes.c_double), ("p_inf", ctypes.c_double)]


class SSDError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"SSD error {code}: {msg}")
        self.code = code


_lib = None


def build(force: bool = False) -> str:
    return _build_mod.build(force=force, debug=_DEBUG)


def lib():
    """Load libssd.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build the CUDA library first (build())")
        L = ctypes.CDLL(LIB_PATH)
        vp = ctypes.c_void_p
        L.sd_create.argtypes = [ctypes.POINTER(sd_mesh), ctypes.c_int, ctypes.POINTER(sd_params),
                                ctypes.POINTER(vp)]
        L.sd_create_error.restype = ctypes.c_char_p
        L.sd_destroy.argtypes = [vp]
        L.sd_last_error.argtypes = [vp]
        L.sd_last_error.restype = ctypes.c_char_p
        L.sd_info.argtypes = [vp, _c_int_p, _c_int_p, ctypes.POINTER(ctypes.c_longlong)]
        L.sd_set_state.argtypes = [vp, vp, ctypes.c_int]
        L.sd_get_state.argtypes = [vp, vp, ctypes.c_int]
        L.sd_set_time.argtypes = [vp, ctypes.c_double]
        L.sd_get_time.argtypes = [vp, _c_dbl_p]
        L.sd_residual.argtypes = [vp, vp, ctypes.c_int]
        L.sd_step.argtypes = [vp, ctypes.c_double, ctypes.c_int]
        L.sd_sync.argtypes = [vp]
        L.sd_sp_coords.argtypes = [vp, ctypes.c_double, vp, ctypes.c_int]
        L.sd_profile_step.argtypes = [vp, ctypes.c_double, ctypes.c_int, _c_dbl_p]
        L.sd_fma_peak.argtypes = [vp, ctypes.c_int, _c_dbl_p]
        L.sd_residual_noalloc.argtypes = [vp, vp, ctypes.c_int]
        L.sd_test_wait_timeout.argtypes = [vp, ctypes.c_int]
        L.sd_test_reciprocal.argtypes = [vp, _c_dbl_p, _c_dbl_p, ctypes.c_int]
        L.sd_batch_create.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.POINTER(sd_mesh)), _c_int_p,
                                      ctypes.POINTER(sd_params), ctypes.c_double, ctypes.POINTER(vp)]
        L.sd_batch_destroy.argtypes = [vp]
        L.sd_batch_size.argtypes = [vp]
        L.sd_batch_case.argtypes = [vp, ctypes.c_int]
        L.sd_batch_case.restype = vp
        L.sd_batch_step.argtypes = [vp, _c_dbl_p, ctypes.c_int]
        L.sd_batch_sync.argtypes = [vp]
        L.sd_batch_last_error.argtypes = [vp]
        L.sd_batch_last_error.restype = ctypes.c_char_p
        L.sd_batch_classes.argtypes = [vp]
        L.sd_batch_class_info.argtypes = [vp, ctypes.c_int, _c_int_p]
        _lib = L
    return _lib


def _ptr(a, dtype, count=None, device=None):
    """(pointer, on_device) for a numpy array or a torch tensor; with ``count``
    the buffer must hold exactly that many values, and a CUDA tensor must
    live on ``device`` (the handle's device) when that is given."""
    if isinstance(a, np.ndarray):
        if a.dtype != dtype or not a.flags["C_CONTIGUOUS"]:
            raise ValueError(f"need a C-contiguous {dtype} array")
        if count is not None and a.size != count:
            raise ValueError(f"need {count} values, got {a.size}")
        return ctypes.c_void_p(a.ctypes.data), 0
    # torch tensor
    if not a.is_contiguous() or str(a.dtype) != "torch.float64":
        raise ValueError("need a contiguous float64 tensor")
    if count is not None and a.numel() != count:
        raise ValueError(f"need {count} values, got {a.numel()}")
    if a.is_cuda and device is not None and a.device.index != device:
        raise ValueError(f"tensor on cuda:{a.device.index}, the solver on cuda:{device}")
    return ctypes.c_void_p(a.data_ptr()), 1 if a.is_cuda else 0


def _current_device():
    """The CUDA device current at handle creation (the handle's device), or
    None when torch is not loaded."""
    import sys
    torch = sys.modules.get("torch")
    if torch is None:
        return None
    try:
        return torch.cuda.current_device() if torch.cuda.is_available() else None
    except Exception:
        return None


def _mesh_struct(mesh: dict, keep: list) -> sd_mesh:
    def arr(x, dt):
        a = np.ascontiguousarray(x, dtype=dt)
        keep.append(a)
        return a

    xy = arr(mesh["xy"], np.float64)
    en = arr(mesh["elem_nodes"], np.int32)
    zone = arr(mesh["elem_zone"], np.int32)
    arc = arr(mesh["edge_arc"], np.int32)
    bf = arr(mesh["bfaces"], np.int32)
    pf = arr(mesh["pfaces"], np.int32)
    Lf = arr(mesh["ifaces_L"], np.int32)
    Rf = arr(mesh["ifaces_R"], np.int32)
    enode = arr(mesh["edge_nodes"], np.int32) if "edge_nodes" in mesh else None
    azone = arr(mesh["elem_arc_zone"], np.int32) if "elem_arc_zone" in mesh else None

    def ip(a):
        return a.ctypes.data_as(_c_int_p)

    # further rotating zones 2, 3, ... (each with its own interface)
    extra = mesh.get("zones", [])
    zones = (sd_zone * max(len(extra), 1))()
    keep.append(zones)
    for k, z in enumerate(extra):
        zl, zr = arr(z["ifaces_L"], np.int32).reshape(-1, 2), arr(z["ifaces_R"], np.int32).reshape(-1, 2)
        zones[k] = sd_zone((ctypes.c_double * 2)(float(z["center"][0]), float(z["center"][1])),
                           float(z["r_interface"]), float(z["omega"]), len(zl), ip(zl), len(zr), ip(zr))
    return sd_mesh(len(xy), xy.ctypes.data_as(_c_dbl_p), len(en), ip(en), ip(zone), ip(arc), len(bf), ip(bf),
                   len(pf), ip(pf), len(Lf), ip(Lf), len(Rf), ip(Rf),
                   (ctypes.c_double * 2)(float(mesh["center"][0]), float(mesh["center"][1])),
                   float(mesh["r_interface"]), ip(enode) if enode is not None else None, len(extra),
                   zones, ip(azone) if azone is not None else None)


def _params_struct(params, precision, stream=None) -> sd_params:
    return sd_params(params.gamma, params.Rgas, params.mu, params.prandtl, params.omega, params.T_wall,
                     int(params.viscous), int(precision), ctypes.c_void_p(stream) if stream else None,
                     int(getattr(params, "rk_stages", 3)), float(getattr(params, "rho_inf", 1.0)),
                     float(getattr(params, "u_inf", 0.0)), float(getattr(params, "v_inf", 0.0)),
                     float(getattr(params, "p_inf", 1.0)))


class Solver:
    """Owns one sd_handle (or wraps a batch's case); methods mirror the C ABI names."""

    @classmethod
    def _wrap(cls, handle, owner):
        self = cls.__new__(cls)
        self._h = ctypes.c_void_p(handle)
        self._owner = owner
        self._owned = False
        self._init_sizes()
        return self

    def _init_sizes(self):
        E, N, n = ctypes.c_int(), ctypes.c_int(), ctypes.c_longlong()
        lib().sd_info(self._h, ctypes.byref(E), ctypes.byref(N), ctypes.byref(n))
        self.E, self.N, self.n_dofs = E.value, N.value, n.value
        self.p = self.N - 1
        self.shape = (self.E, 4, self.N, self.N)
        self.device = _current_device()

    def _state_ptr(self, a):
        return _ptr(a, np.float64, self.n_dofs, self.device)

    def __init__(self, mesh: dict, p: int, params, precision: int = SD_PREC_FP64, stream=None):
        L = lib()
        self._keep = []
        self._owned = True
        m = _mesh_struct(mesh, self._keep)
        prm = _params_struct(params, precision, stream)
        h = ctypes.c_void_p()
        rc = L.sd_create(ctypes.byref(m), p, ctypes.byref(prm), ctypes.byref(h))
        if rc != SD_OK:
            raise SSDError(rc, L.sd_create_error().decode())
        self._h = h
        self._init_sizes()

    def _check(self, rc):
        if rc != SD_OK:
            raise SSDError(rc, lib().sd_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None) and getattr(self, "_owned", True):
            lib().sd_destroy(self._h)
        self._h = None

    def __del__(self):
        self.close()

    def sd_set_state(self, Q):
        p, dev = self._state_ptr(Q)
        self._check(lib().sd_set_state(self._h, p, dev))

    def sd_get_state(self, out=None):
        if out is None:
            out = np.empty(self.shape)
        p, dev = self._state_ptr(out)
        self._check(lib().sd_get_state(self._h, p, dev))
        return out

    def sd_set_time(self, t):
        self._check(lib().sd_set_time(self._h, float(t)))

    def sd_get_time(self):
        t = ctypes.c_double()
        self._check(lib().sd_get_time(self._h, ctypes.byref(t)))
        return t.value

    def sd_residual(self, out=None):
        if out is None:
            out = np.empty(self.shape)
        p, dev = self._state_ptr(out)
        self._check(lib().sd_residual(self._h, p, dev))
        return out

    def sd_residual_noalloc(self, out=None):
        """sd_residual without any device allocation (fixed 16 MiB work memory
        inside the library); ``out`` must be preallocated by a caller that
        cannot allocate, or is created here in host memory."""
        if out is None:
            out = np.empty(self.shape)
        p, dev = self._state_ptr(out)
        self._check(lib().sd_residual_noalloc(self._h, p, dev))
        return out

    def sd_step(self, dt, nsteps=1):
        self._check(lib().sd_step(self._h, float(dt), int(nsteps)))

    def sd_sync(self):
        self._check(lib().sd_sync(self._h))

    def sd_test_wait_timeout(self, on):
        self._check(lib().sd_test_wait_timeout(self._h, int(on)))

    def sd_test_reciprocal(self, x):
        """1 / x in the handle's compute type, on the GPU (test aid)."""
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.empty_like(x)
        self._check(lib().sd_test_reciprocal(self._h, x.ctypes.data_as(_c_dbl_p), y.ctypes.data_as(_c_dbl_p),
                                              int(x.size)))
        return y

    def sd_sp_coords(self, t=0.0, out=None):
        if out is None:
            out = np.empty((self.E, self.N, self.N, 2))
        p, dev = _ptr(out, np.float64, self.E * self.N * self.N * 2, self.device)
        self._check(lib().sd_sp_coords(self._h, float(t), p, dev))
        return out

    def sd_profile_step(self, dt, reps=1):
        ms = (ctypes.c_double * 5)()
        self._check(lib().sd_profile_step(self._h, float(dt), int(reps), ms))
        return {"merge": ms[0], "faces": ms[1], "mortar": ms[2], "volume": ms[3], "step": ms[4]}

    def sd_fma_peak(self, precision):
        v = ctypes.c_double()
        self._check(lib().sd_fma_peak(self._h, int(precision), ctypes.byref(v)))
        return v.value

    def state_from(self, field_fn, t=0.0):
        xy = self.sd_sp_coords(t)
        return np.ascontiguousarray(np.moveaxis(field_fn(xy[..., 0], xy[..., 1]), -1, 1))


class Batch:
    """Owns one sd_batch: independent cases (mesh, p, params each) advanced
    together with one CUDA-graph launch per step."""

    def __init__(self, meshes, ps, params, precision=SD_PREC_FP64, tune_dt=0.0):
        L = lib()
        n = len(meshes)
        self._keep = []
        structs = [_mesh_struct(m, self._keep) for m in meshes]
        self._keep.append(structs)
        mptrs = (ctypes.POINTER(sd_mesh) * n)(*[ctypes.pointer(x) for x in structs])
        parr = (ctypes.c_int * n)(*[int(p) for p in ps])
        prms = (sd_params * n)(*[_params_struct(pr, precision) for pr in params])
        b = ctypes.c_void_p()
        rc = L.sd_batch_create(n, mptrs, parr, prms, float(tune_dt), ctypes.byref(b))
        if rc != SD_OK:
            raise SSDError(rc, L.sd_create_error().decode())
        self._b = b
        self.cases = [Solver._wrap(L.sd_batch_case(b, i), self) for i in range(n)]

    def close(self):
        if getattr(self, "_b", None):
            for c in self.cases:
                c._h = None
            lib().sd_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        self.close()

    def _check(self, rc):
        if rc != SD_OK:
            raise SSDError(rc, lib().sd_batch_last_error(self._b).decode())

    def sd_batch_step(self, dts, nsteps=1):
        arr = (ctypes.c_double * len(self.cases))(*[float(d) for d in dts])
        self._check(lib().sd_batch_step(self._b, arr, int(nsteps)))

    def sd_batch_sync(self):
        self._check(lib().sd_batch_sync(self._b))

    def class_info(self):
        """Per class of cases (equal N and viscous flag): its size and the
        launch shapes in force (the autotuner's choice)."""
        out = []
        for i in range(lib().sd_batch_classes(self._b)):
            info = (ctypes.c_int * 6)()
            self._check(lib().sd_batch_class_info(self._b, i, info))
            out.append({"N": info[0], "viscous": info[1], "cases": info[2], "tile_elems": info[3],
                        "vol_ctas_per_sm": info[4], "face_block": info[5]})
        return out
