"""Plain FP64 CPU oracle of the DG-SWEM hot path (ctypes wrapper over dgswem_oracle.c).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product
(``paper_2508_21208_gb300``) never imports it, and the two share no code.

The C source follows the paper's Sec. 2 (model and DG formulation) and
Algorithms 1-3 (AREA, EDGE, GATHER); see its header for the readings taken
where the paper is silent.  Partly pinned: the slope limiter and the wet/dry
treatment are checked through invariants and hand-worked examples (the limiter
also against a recomputation from the mesh geometry, wet/dry also against
Thacker's moving-shoreline solution in a parabolic bowl).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dgswem_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIBS = {}


def build(force: bool = False) -> None:
    """Compile the oracle twice: single-threaded and with OpenMP (same source)."""
    os.makedirs(_BUILD, exist_ok=True)
    for name, extra in (("liboracle.so", []), ("liboracle_omp.so", ["-fopenmp"])):
        out = os.path.join(_BUILD, name)
        if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
            continue
        cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fPIC", "-shared", *extra,
               "-o", out, _SRC, "-lm"]
        subprocess.run(cmd, check=True)


class Params(C.Structure):
    _fields_ = [("p", C.c_int32), ("g", C.c_double), ("cfl", C.c_double), ("dt", C.c_double),
                ("h0", C.c_double), ("friction", C.c_int32), ("manning_n", C.c_double),
                ("cf", C.c_double), ("limiter", C.c_int32), ("coriolis", C.c_int32),
                ("coriolis_lat_deg", C.c_double), ("tide_amp", C.c_double),
                ("tide_period", C.c_double), ("tide_phase", C.c_double), ("hurricane", C.c_int32),
                ("pc_hpa", C.c_double), ("pn_hpa", C.c_double), ("rmax_m", C.c_double),
                ("holland_b", C.c_double), ("vt_ms", C.c_double), ("track_x0", C.c_double),
                ("track_y0", C.c_double), ("track_heading", C.c_double), ("rho_air", C.c_double),
                ("rho_water", C.c_double), ("rk_scheme", C.c_int32), ("rk_stages", C.c_int32),
                ("rk_coeffs", C.c_double * 24), ("flux", C.c_int32), ("rain_rate", C.c_double),
                ("river_q", C.c_double)]


FIELD_CB = C.CFUNCTYPE(None, C.c_double, C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_double))
_dp = C.POINTER(C.c_double)


def _lib(omp: bool = False):
    key = "omp" if omp else "serial"
    if key in _LIBS:
        return _LIBS[key]
    build()
    lib = C.CDLL(os.path.join(_BUILD, "liboracle_omp.so" if omp else "liboracle.so"))
    lib.orc_create.restype = C.c_void_p
    lib.orc_create.argtypes = [C.c_int32, C.c_int32, _dp, C.POINTER(C.c_int32), C.c_int32,
                               C.POINTER(C.c_int32), C.POINTER(C.c_int32), _dp, C.POINTER(Params),
                               _dp, _dp, C.c_double]
    lib.orc_destroy.argtypes = [C.c_void_p]
    lib.orc_sizes.argtypes = [C.c_void_p, C.POINTER(C.c_int32)]
    lib.orc_step.argtypes = [C.c_void_p, C.c_int32]
    lib.orc_stage.argtypes = [C.c_void_p]
    lib.orc_stage.restype = C.c_int32
    lib.orc_stage_count.argtypes = [C.c_void_p]
    lib.orc_stage_count.restype = C.c_int32
    lib.orc_get_register.argtypes = [C.c_void_p, C.c_int32, _dp, _dp, _dp]
    lib.orc_set_register.argtypes = [C.c_void_p, C.c_int32, _dp, _dp, _dp]
    lib.orc_set_flags.argtypes = [C.c_void_p, C.POINTER(C.c_uint8)]
    lib.orc_get_state.argtypes = [C.c_void_p, _dp, _dp, _dp]
    lib.orc_set_state.argtypes = [C.c_void_p, _dp, _dp, _dp, C.c_double]
    lib.orc_info.argtypes = [C.c_void_p, _dp, _dp, C.POINTER(C.c_int64)]
    lib.orc_mass.argtypes = [C.c_void_p, _dp, _dp]
    lib.orc_rhs.argtypes = [C.c_void_p, C.c_double, _dp]
    lib.orc_apply_limiter.argtypes = [C.c_void_p]
    lib.orc_apply_wetdry.argtypes = [C.c_void_p]
    lib.orc_flags.argtypes = [C.c_void_p, C.POINTER(C.c_uint8)]
    lib.orc_forcing.argtypes = [C.c_void_p, C.c_double, _dp]
    lib.orc_basis.argtypes = [C.c_int32, C.c_double, C.c_double, _dp, _dp, _dp]
    lib.orc_area_rule.argtypes = [C.c_int32, _dp, _dp, _dp]
    lib.orc_area_rule.restype = C.c_int32
    lib.orc_high_rule.argtypes = [_dp, _dp, _dp]
    lib.orc_high_rule.restype = C.c_int32
    lib.orc_edge_rule.argtypes = [C.c_int32, _dp, _dp]
    lib.orc_edge_rule.restype = C.c_int32
    lib.orc_set_mms.argtypes = [C.c_void_p, FIELD_CB, FIELD_CB]
    lib.orc_project.argtypes = [C.c_void_p, FIELD_CB, C.c_double]
    lib.orc_set_transmissive.argtypes = [C.c_void_p, C.c_int32]
    lib.orc_numflux.argtypes = [C.POINTER(Params), _dp, _dp, C.c_double, C.c_double, C.c_double, _dp]
    lib.orc_l2err.argtypes = [C.c_void_p, FIELD_CB, C.c_double, _dp]
    _LIBS[key] = lib
    return lib


def _ptr(a, ct=C.c_double):
    return a.ctypes.data_as(C.POINTER(ct))


def make_params(d: dict) -> Params:
    prm = Params()
    for name, _ in Params._fields_:
        if name == "rk_coeffs":
            vals = list(d.get(name) or [])
            prm.rk_coeffs = (C.c_double * 24)(*(vals + [0.0] * (24 - len(vals))))
        else:
            setattr(prm, name, d[name])
    return prm


def _field_cb(fn):
    """Wrap fn(t, xy[n,2]) -> values[n,3] as a C callback."""
    def cb(t, n, xy, out):
        X = np.ctypeslib.as_array(xy, shape=(n, 2))
        O = np.ctypeslib.as_array(out, shape=(n, 3))
        O[:] = fn(t, X)
    return FIELD_CB(cb)


class Oracle:
    """One oracle model: a mesh, nodal bathymetry, parameters and a state."""

    def __init__(self, mesh, bathy, params: dict, init_nodal=None, init_modal=None, t0=0.0,
                 omp: bool = False):
        self.lib = _lib(omp)
        self.mesh = mesh
        self._keep = dict(xy=np.ascontiguousarray(mesh.xy, np.float64),
                          tri=np.ascontiguousarray(mesh.tri, np.int32),
                          be=np.ascontiguousarray(mesh.bedge, np.int32).reshape(-1),
                          bt=np.ascontiguousarray(mesh.bedge_type, np.int32),
                          hb=np.ascontiguousarray(bathy, np.float64))
        k = self._keep
        self.prm = make_params(params)
        nodal = None if init_nodal is None else np.ascontiguousarray(init_nodal, np.float64)
        modal = None if init_modal is None else np.ascontiguousarray(init_modal, np.float64)
        self.h = self.lib.orc_create(mesh.n_nodes, mesh.n_elems, _ptr(k["xy"]), _ptr(k["tri"], C.c_int32),
                                     len(k["bt"]), _ptr(k["be"], C.c_int32), _ptr(k["bt"], C.c_int32),
                                     _ptr(k["hb"]), C.byref(self.prm),
                                     _ptr(nodal) if nodal is not None else None,
                                     _ptr(modal) if modal is not None else None, float(t0))
        if not self.h:
            raise ValueError("oracle: invalid mesh or parameters")
        sz = (C.c_int32 * 5)()
        self.lib.orc_sizes(self.h, sz)
        self.nd, self.nqa, self.nqe, self.n_edges, self.n_interior = list(sz)
        self.ne = mesh.n_elems
        self._cbs = []

    def __del__(self):
        if getattr(self, "h", None):
            self.lib.orc_destroy(self.h)
            self.h = None

    def step(self, n: int = 1):
        self.lib.orc_step(self.h, int(n))

    def stage(self) -> int:
        """Advance one stage of the time step in progress; returns the state buffer it wrote."""
        return int(self.lib.orc_stage(self.h))

    def stage_count(self) -> int:
        return int(self.lib.orc_stage_count(self.h))

    def register(self, r: int) -> np.ndarray:
        out = np.empty((3, self.nd, self.ne))
        self.lib.orc_get_register(self.h, int(r), _ptr(out[0]), _ptr(out[1]), _ptr(out[2]))
        return out

    def set_register(self, r: int, u):
        u = np.ascontiguousarray(u, np.float64)
        self.lib.orc_set_register(self.h, int(r), _ptr(u[0]), _ptr(u[1]), _ptr(u[2]))

    def set_flags(self, f):
        f = np.ascontiguousarray(f, np.uint8)
        self.lib.orc_set_flags(self.h, _ptr(f, C.c_uint8))

    def state(self) -> np.ndarray:
        out = np.empty((3, self.nd, self.ne))
        self.lib.orc_get_state(self.h, _ptr(out[0]), _ptr(out[1]), _ptr(out[2]))
        return out

    def set_state(self, u, t=0.0):
        u = np.ascontiguousarray(u, np.float64)
        self.lib.orc_set_state(self.h, _ptr(u[0]), _ptr(u[1]), _ptr(u[2]), float(t))

    def info(self):
        dt, t, s = C.c_double(), C.c_double(), C.c_int64()
        self.lib.orc_info(self.h, C.byref(dt), C.byref(t), C.byref(s))
        return dt.value, t.value, s.value

    @property
    def dt(self):
        return self.info()[0]

    def mass(self):
        m, v = C.c_double(), C.c_double()
        self.lib.orc_mass(self.h, C.byref(m), C.byref(v))
        return m.value, v.value

    def rhs(self, t: float) -> np.ndarray:
        out = np.empty((3, self.nd, self.ne))
        self.lib.orc_rhs(self.h, float(t), _ptr(out))
        return out

    def apply_limiter(self):
        self.lib.orc_apply_limiter(self.h)

    def apply_wetdry(self):
        self.lib.orc_apply_wetdry(self.h)

    def flags(self) -> np.ndarray:
        out = np.empty(self.ne, np.uint8)
        self.lib.orc_flags(self.h, _ptr(out, C.c_uint8))
        return out

    def forcing(self, t: float) -> np.ndarray:
        out = np.empty((3, self.mesh.n_nodes))
        self.lib.orc_forcing(self.h, float(t), _ptr(out))
        return out

    def set_mms(self, src_fn, bnd_fn):
        cbs = (_field_cb(src_fn), _field_cb(bnd_fn))
        self._cbs.append(cbs)
        self.lib.orc_set_mms(self.h, cbs[0], cbs[1])

    def set_transmissive(self, on=True):
        self.lib.orc_set_transmissive(self.h, 1 if on else 0)

    def project(self, fn, t=0.0):
        cb = _field_cb(fn)
        self.lib.orc_project(self.h, cb, float(t))

    def l2err(self, fn, t):
        cb = _field_cb(fn)
        out = (C.c_double * 3)()
        self.lib.orc_l2err(self.h, cb, float(t), out)
        return np.array(list(out))


def numflux(params: dict, wi, wo, hb, nx, ny):
    lib = _lib()
    prm = make_params(params)
    a, b = np.ascontiguousarray(wi, np.float64), np.ascontiguousarray(wo, np.float64)
    out = np.zeros(3)
    lib.orc_numflux(C.byref(prm), _ptr(a), _ptr(b), float(hb), float(nx), float(ny), _ptr(out))
    return out


def basis(p: int, xi: float, eta: float):
    lib = _lib()
    ph, dx, dy = (np.zeros(6) for _ in range(3))
    lib.orc_basis(p, xi, eta, _ptr(ph), _ptr(dx), _ptr(dy))
    n = (p + 1) * (p + 2) // 2
    return ph[:n], dx[:n], dy[:n]


def area_rule(p: int):
    lib = _lib()
    a, b, w = (np.zeros(16) for _ in range(3))
    n = lib.orc_area_rule(p, _ptr(a), _ptr(b), _ptr(w))
    return a[:n], b[:n], w[:n]


def high_rule():
    lib = _lib()
    a, b, w = (np.zeros(64) for _ in range(3))
    n = lib.orc_high_rule(_ptr(a), _ptr(b), _ptr(w))
    return a[:n], b[:n], w[:n]


def edge_rule(n: int):
    lib = _lib()
    s, w = np.zeros(n), np.zeros(n)
    lib.orc_edge_rule(n, _ptr(s), _ptr(w))
    return s, w
