"""Thin Python binding of libdgswem.so (argument marshalling only).

Every step of the hot path runs in the library's CUDA kernels; this module converts numpy arrays
to the C structures of include/dgswem.h, and takes the one device workspace and the CUDA stream
from PyTorch.  There is no CPU fallback: if the library or a GPU is missing, construction fails.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdgswem.so")

DGSWEM_OK = 0
ERRORS = {-1: "EINVAL", -2: "EMESH", -3: "ECUDA", -4: "ENONFINITE", -5: "ENEGDEPTH", -6: "ETIMEOUT",
          -7: "ENOMEM", -8: "ESTATE", -9: "ETOOBIG"}
VARIANT_AUTO, VARIANT_SPLIT, VARIANT_FUSED, VARIANT_TILED, VARIANT_TILED_WIDE = 0, 1, 2, 3, 4
ENSEMBLE_PERSISTENT, ENSEMBLE_PHASED = 1, 2
FLUX_LLF, FLUX_ROE = 0, 1
FP64, FP32_MIXED = 0, 1


class DgswemError(RuntimeError):
    def __init__(self, code, msg=""):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Mesh(C.Structure):
    _fields_ = [("n_nodes", C.c_int32), ("n_elems", C.c_int32), ("n_bedges", C.c_int32),
                ("xy", C.POINTER(C.c_double)), ("tri", C.POINTER(C.c_int32)),
                ("bedge", C.POINTER(C.c_int32)), ("bedge_type", C.POINTER(C.c_int32))]


class Params(C.Structure):
    _fields_ = [("p", C.c_int32), ("precision", C.c_int32), ("g", C.c_double), ("cfl", C.c_double),
                ("dt", C.c_double), ("h0", C.c_double), ("friction", C.c_int32),
                ("manning_n", C.c_double), ("cf", C.c_double), ("limiter", C.c_int32),
                ("coriolis", C.c_int32), ("coriolis_lat_deg", C.c_double), ("tide_amp", C.c_double),
                ("tide_period", C.c_double), ("tide_phase", C.c_double), ("hurricane", C.c_int32),
                ("pc_hpa", C.c_double), ("pn_hpa", C.c_double), ("rmax_m", C.c_double),
                ("holland_b", C.c_double), ("vt_ms", C.c_double), ("track_x0", C.c_double),
                ("track_y0", C.c_double), ("track_heading", C.c_double), ("rho_air", C.c_double),
                ("rho_water", C.c_double), ("rk_scheme", C.c_int32), ("rk_stages", C.c_int32),
                ("rk_coeffs", C.c_double * 24), ("flux", C.c_int32), ("rain_rate", C.c_double),
                ("river_q", C.c_double)]


class Tuning(C.Structure):
    _fields_ = [("variant", C.c_int32), ("block", C.c_int32), ("reorder", C.c_int32),
                ("autotune", C.c_int32)]


class PartCounts(C.Structure):
    _fields_ = [(n, C.c_int32) for n in ("n_nodes", "n_elems", "n_bedges", "n_own", "n_ghost1", "n_ghost2",
                                          "n_peers", "n_send", "n_recv")]


class PartOut(C.Structure):
    _fields_ = [("xy", C.POINTER(C.c_double)), ("tri", C.POINTER(C.c_int32)), ("bedge", C.POINTER(C.c_int32)),
                ("bedge_type", C.POINTER(C.c_int32)), ("bathy", C.POINTER(C.c_double)),
                ("elem_global", C.POINTER(C.c_int32)), ("elem_class", C.POINTER(C.c_int32)),
                ("node_global", C.POINTER(C.c_int32)), ("peer", C.POINTER(C.c_int32)),
                ("send_count", C.POINTER(C.c_int32)), ("recv_count", C.POINTER(C.c_int32)),
                ("send_elems", C.POINTER(C.c_int32)), ("recv_elems", C.POINTER(C.c_int32))]


class Init(C.Structure):
    _fields_ = [("modal", C.POINTER(C.c_double)), ("nodal", C.POINTER(C.c_double)), ("t0", C.c_double)]


class PartSpec(C.Structure):
    _fields_ = [("elem_class", C.POINTER(C.c_int32)), ("n_send", C.c_int32), ("send_elems", C.POINTER(C.c_int32)),
                ("n_recv", C.c_int32), ("recv_elems", C.POINTER(C.c_int32))]


_dp = C.POINTER(C.c_double)
_vp = C.c_void_p
_lib = None

# (name, restype, argtypes) of every entry point in include/dgswem.h
SIGNATURES = [
    ("dgswem_create", C.c_int, [C.POINTER(Mesh), _dp, C.POINTER(Params), C.POINTER(Init), C.POINTER(Tuning),
                                C.POINTER(_vp)]),
    ("dgswem_workspace_size", C.c_int, [_vp, C.POINTER(C.c_size_t)]),
    ("dgswem_attach", C.c_int, [_vp, _vp, C.c_size_t, _vp]),
    ("dgswem_step", C.c_int, [_vp, C.c_int32]),
    ("dgswem_get_state", C.c_int, [_vp, _dp, _dp, _dp]),
    ("dgswem_set_state", C.c_int, [_vp, _dp, _dp, _dp, C.c_double]),
    ("dgswem_mass", C.c_int, [_vp, _dp, _dp]),
    ("dgswem_info", C.c_int, [_vp, _dp, _dp, C.POINTER(C.c_int64)]),
    ("dgswem_sync", C.c_int, [_vp]),
    ("dgswem_get_flags", C.c_int, [_vp, C.POINTER(C.c_uint8)]),
    ("dgswem_destroy", None, [_vp]),
    ("dgswem_last_error", C.c_char_p, [_vp]),
    ("dgswem_eval_rhs", C.c_int, [_vp, C.c_double, _dp]),
    ("dgswem_apply_limiter", C.c_int, [_vp]),
    ("dgswem_apply_wetdry", C.c_int, [_vp]),
    ("dgswem_eval_forcing", C.c_int, [_vp, C.c_double, _dp]),
    ("dgswem_set_kernel_timing", C.c_int, [_vp, C.c_int32]),
    ("dgswem_kernel_times", C.c_int, [_vp, C.POINTER(C.c_float), C.POINTER(C.c_char_p), C.c_int32,
                                      C.POINTER(C.c_int32)]),
    ("dgswem_graph_info", C.c_int, [_vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    ("dgswem_tune_log", C.c_int, [_vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_float), C.c_int32,
                                  C.POINTER(C.c_int32)]),
    ("dgswem_ensemble_create", C.c_int, [C.c_int32, C.POINTER(C.POINTER(Mesh)), C.POINTER(_dp),
                                         C.POINTER(Params), C.POINTER(Init), C.POINTER(Tuning), C.POINTER(_vp)]),
    ("dgswem_ensemble_step", C.c_int, [_vp, C.c_int32]),
    ("dgswem_ensemble_get_state", C.c_int, [_vp, C.c_int32, _dp, _dp, _dp]),
    ("dgswem_ensemble_get_flags", C.c_int, [_vp, C.c_int32, C.POINTER(C.c_uint8)]),
    ("dgswem_ensemble_info", C.c_int, [_vp, C.c_int32, _dp, _dp, C.POINTER(C.c_int64)]),
    ("dgswem_ensemble_set_fault", C.c_int, [_vp, C.c_int32]),
    ("dgswem_mass_noalloc", C.c_int, [_vp, _vp, _vp, C.c_int32, _vp, _vp]),
    ("dgswem_partition_rcb", C.c_int, [C.POINTER(Mesh), C.c_int32, C.POINTER(C.c_int32)]),
    ("dgswem_part_sizes", C.c_int, [C.POINTER(Mesh), C.POINTER(C.c_int32), C.c_int32, C.c_int32,
                                    C.POINTER(PartCounts)]),
    ("dgswem_part_build", C.c_int, [C.POINTER(Mesh), _dp, C.POINTER(C.c_int32), C.c_int32, C.c_int32,
                                    C.POINTER(PartOut)]),
    ("dgswem_create_part", C.c_int, [C.POINTER(Mesh), _dp, C.POINTER(Params), C.POINTER(Init), C.POINTER(Tuning),
                                     C.POINTER(PartSpec), C.POINTER(_vp)]),
    ("dgswem_halo_sizes", C.c_int, [_vp, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)]),
    ("dgswem_halo_attach", C.c_int, [_vp, _vp, _vp]),
    ("dgswem_stage_compute", C.c_int, [_vp]),
    ("dgswem_stage_finish", C.c_int, [_vp]),
]


def load_library(path: str = LIB_PATH):
    """Load libdgswem.so; raises if it has not been built (no fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_2508_21208_gb300.build.build_library()")
    lib = C.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(a, ct=C.c_double):
    return a.ctypes.data_as(C.POINTER(ct)) if a is not None else None


def _torch_cuda():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("libdgswem needs a CUDA GPU; none is visible")
    return torch


def make_params(d: dict) -> Params:
    p = Params()
    for name, _ in Params._fields_:
        if name == "rk_coeffs":
            vals = list(d.get(name) or [])
            p.rk_coeffs = (C.c_double * 24)(*(vals + [0.0] * (24 - len(vals))))
        else:
            setattr(p, name, d[name])
    return p


class _MeshArrays:
    """Keeps the contiguous numpy copies alive for the duration of a create call."""

    def __init__(self, mesh):
        self.xy = np.ascontiguousarray(mesh.xy, np.float64)
        self.tri = np.ascontiguousarray(mesh.tri, np.int32)
        self.be = np.ascontiguousarray(mesh.bedge, np.int32).reshape(-1)
        self.bt = np.ascontiguousarray(mesh.bedge_type, np.int32)
        self.s = Mesh(mesh.n_nodes, mesh.n_elems, len(self.bt), _ptr(self.xy), _ptr(self.tri, C.c_int32),
                      _ptr(self.be, C.c_int32), _ptr(self.bt, C.c_int32))


class _Handle:
    def __init__(self):
        self.lib = load_library()
        self.h = _vp()
        self._ws = None

    def _check(self, rc):
        if rc != DGSWEM_OK:
            msg = self.lib.dgswem_last_error(self.h).decode() if self.h else ""
            raise DgswemError(rc, msg)

    def _attach(self, stream=None):
        torch = _torch_cuda()
        n = C.c_size_t()
        self._check(self.lib.dgswem_workspace_size(self.h, C.byref(n)))
        # one device workspace from PyTorch's allocator (256-byte aligned); the library allocates none
        self._ws = torch.empty(max(int(n.value), 1) + 256, dtype=torch.uint8, device="cuda")
        base = self._ws.data_ptr()
        aligned = (base + 255) // 256 * 256
        s = stream if stream is not None else torch.cuda.current_stream()
        self.stream = s
        self._check(self.lib.dgswem_attach(self.h, _vp(aligned), int(n.value), _vp(s.cuda_stream)))

    def close(self):
        if self.h:
            self.lib.dgswem_destroy(self.h)
            self.h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n: int = 1):
        self._check(self.lib.dgswem_step(self.h, int(n)))

    def sync(self):
        self._check(self.lib.dgswem_sync(self.h))

    def graph_info(self):
        k, v, b = C.c_int32(), C.c_int32(), C.c_int32()
        self._check(self.lib.dgswem_graph_info(self.h, C.byref(k), C.byref(v), C.byref(b)))
        return k.value, v.value, b.value

    def tune_log(self):
        cap = 64
        v, b, ms = (C.c_int32 * cap)(), (C.c_int32 * cap)(), (C.c_float * cap)()
        n = C.c_int32()
        self._check(self.lib.dgswem_tune_log(self.h, v, b, ms, cap, C.byref(n)))
        return [(int(v[i]), int(b[i]), float(ms[i])) for i in range(min(n.value, cap))]

    def set_kernel_timing(self, on: bool):
        self._check(self.lib.dgswem_set_kernel_timing(self.h, 1 if on else 0))

    def kernel_times(self):
        cap = 32
        ms = (C.c_float * cap)()
        names = (C.c_char_p * cap)()
        n = C.c_int32()
        self._check(self.lib.dgswem_kernel_times(self.h, ms, names, cap, C.byref(n)))
        return [(names[i].decode(), float(ms[i])) for i in range(n.value)]


class Model(_Handle):
    """One DG-SWEM model on the current CUDA device (dgswem_create + dgswem_attach)."""

    def __init__(self, mesh, bathy, params: dict, init_nodal=None, init_modal=None, t0=0.0, variant=0,
                 block=0, reorder=0, stream=None):
        super().__init__()
        m = _MeshArrays(mesh)
        hb = np.ascontiguousarray(bathy, np.float64)
        self.prm = make_params(params)
        nodal = None if init_nodal is None else np.ascontiguousarray(init_nodal, np.float64)
        modal = None if init_modal is None else np.ascontiguousarray(init_modal, np.float64)
        ini = Init(_ptr(modal), _ptr(nodal), float(t0))
        tun = Tuning(int(variant), int(block), int(reorder), 0)
        rc = self.lib.dgswem_create(C.byref(m.s), _ptr(hb), C.byref(self.prm), C.byref(ini), C.byref(tun),
                                    C.byref(self.h))
        if rc != DGSWEM_OK:
            raise DgswemError(rc, "dgswem_create")
        self.ne = mesh.n_elems
        self.nn = mesh.n_nodes
        self.nd = (params["p"] + 1) * (params["p"] + 2) // 2
        self._attach(stream)

    def state(self) -> np.ndarray:
        out = np.empty((3, self.nd, self.ne))
        self._check(self.lib.dgswem_get_state(self.h, _ptr(out[0]), _ptr(out[1]), _ptr(out[2])))
        return out

    def get_state_into(self, z, qx, qy):
        """Copy the state into caller-owned (e.g. pinned) host arrays."""
        self._check(self.lib.dgswem_get_state(self.h, _ptr(z), _ptr(qx), _ptr(qy)))

    def set_state(self, u, t=0.0):
        u = np.ascontiguousarray(u, np.float64)
        self._keep_state = u
        self._check(self.lib.dgswem_set_state(self.h, _ptr(u[0]), _ptr(u[1]), _ptr(u[2]), float(t)))

    def set_state_from(self, z, qx, qy, t=0.0):
        self._check(self.lib.dgswem_set_state(self.h, _ptr(z), _ptr(qx), _ptr(qy), float(t)))

    def mass(self):
        a, b = C.c_double(), C.c_double()
        self._check(self.lib.dgswem_mass(self.h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def info(self):
        dt, t, s = C.c_double(), C.c_double(), C.c_int64()
        self._check(self.lib.dgswem_info(self.h, C.byref(dt), C.byref(t), C.byref(s)))
        return dt.value, t.value, s.value

    @property
    def dt(self):
        return self.info()[0]

    def flags(self) -> np.ndarray:
        out = np.empty(self.ne, np.uint8)
        self._check(self.lib.dgswem_get_flags(self.h, _ptr(out, C.c_uint8)))
        return out

    def eval_rhs(self, t: float) -> np.ndarray:
        out = np.empty((3, self.nd, self.ne))
        self._check(self.lib.dgswem_eval_rhs(self.h, float(t), _ptr(out)))
        return out

    def apply_limiter(self):
        self._check(self.lib.dgswem_apply_limiter(self.h))

    def apply_wetdry(self):
        self._check(self.lib.dgswem_apply_wetdry(self.h))

    def eval_forcing(self, t: float) -> np.ndarray:
        out = np.empty((3, self.nn))
        self._check(self.lib.dgswem_eval_forcing(self.h, float(t), _ptr(out)))
        return out


class Ensemble(_Handle):
    """A batch of scenarios advanced together (dgswem_ensemble_create + dgswem_attach)."""

    def __init__(self, meshes, bathys, members, block=0, mode=0, stream=None):
        """members: list of (mesh_index, params dict, init_nodal or None)."""
        super().__init__()
        marr = [_MeshArrays(m) for m in meshes]
        hbs = [np.ascontiguousarray(b, np.float64) for b in bathys]
        n = len(members)
        mesh_ptrs = (C.POINTER(Mesh) * n)()
        hb_ptrs = (_dp * n)()
        prms = (Params * n)()
        inits = (Init * n)()
        self._keep = []
        for i, (mi, prm, init) in enumerate(members):
            mesh_ptrs[i] = C.pointer(marr[mi].s)
            hb_ptrs[i] = _ptr(hbs[mi])
            prms[i] = make_params(prm)
            nod = None if init is None else np.ascontiguousarray(init, np.float64)
            self._keep.append(nod)
            inits[i] = Init(None, _ptr(nod), 0.0)
        tun = Tuning(int(mode), int(block), 0, 0)
        rc = self.lib.dgswem_ensemble_create(n, mesh_ptrs, hb_ptrs, prms, inits, C.byref(tun), C.byref(self.h))
        if rc != DGSWEM_OK:
            raise DgswemError(rc, "dgswem_ensemble_create")
        self.members = members
        self.meshes = meshes
        self.nd = (members[0][1]["p"] + 1) * (members[0][1]["p"] + 2) // 2
        self._attach(stream)

    def step(self, n: int = 1):
        self._check(self.lib.dgswem_ensemble_step(self.h, int(n)))

    def state(self, i: int) -> np.ndarray:
        ne = self.meshes[self.members[i][0]].n_elems
        out = np.empty((3, self.nd, ne))
        self._check(self.lib.dgswem_ensemble_get_state(self.h, int(i), _ptr(out[0]), _ptr(out[1]), _ptr(out[2])))
        return out

    def flags(self, i: int) -> np.ndarray:
        ne = self.meshes[self.members[i][0]].n_elems
        out = np.empty(ne, np.uint8)
        self._check(self.lib.dgswem_ensemble_get_flags(self.h, int(i), _ptr(out, C.c_uint8)))
        return out

    def info(self, i: int):
        dt, t, s = C.c_double(), C.c_double(), C.c_int64()
        self._check(self.lib.dgswem_ensemble_info(self.h, int(i), C.byref(dt), C.byref(t), C.byref(s)))
        return dt.value, t.value, s.value

    def set_fault(self, on: bool):
        self._check(self.lib.dgswem_ensemble_set_fault(self.h, 1 if on else 0))


# ---------------------------------------------------------------- domain decomposition (Sec. 5.3)
class SubMesh:
    """A part's sub-mesh (the fields _MeshArrays reads)."""

    def __init__(self, xy, tri, bedge, bedge_type):
        self.xy, self.tri, self.bedge, self.bedge_type = xy, tri, bedge, bedge_type

    @property
    def n_nodes(self) -> int:
        return int(self.xy.shape[0])

    @property
    def n_elems(self) -> int:
        return int(self.tri.shape[0])


class Part:
    """dgswem_part_build's output for one part: sub-mesh, bathymetry, global ids, element classes
    and, per peer, the send and receive lists (sub-mesh element indices)."""

    def __init__(self, mesh, bathy, elem_global, elem_class, node_global, peers, send, recv):
        self.mesh, self.bathy = mesh, bathy
        self.elem_global, self.elem_class, self.node_global = elem_global, elem_class, node_global
        self.peers = peers  # list of peer ranks
        self.send = send    # list (per peer) of int32 arrays
        self.recv = recv

    @property
    def send_elems(self):
        return np.concatenate(self.send).astype(np.int32) if self.send else np.zeros(0, np.int32)

    @property
    def recv_elems(self):
        return np.concatenate(self.recv).astype(np.int32) if self.recv else np.zeros(0, np.int32)


def partition_rcb(mesh, n_parts: int) -> np.ndarray:
    lib = load_library()
    m = _MeshArrays(mesh)
    part = np.empty(mesh.n_elems, np.int32)
    rc = lib.dgswem_partition_rcb(C.byref(m.s), int(n_parts), _ptr(part, C.c_int32))
    if rc != DGSWEM_OK:
        raise DgswemError(rc, "dgswem_partition_rcb")
    return part


def build_part(mesh, bathy, part, n_parts: int, rank: int) -> Part:
    lib = load_library()
    m = _MeshArrays(mesh)
    part = np.ascontiguousarray(part, np.int32)
    hb = np.ascontiguousarray(bathy, np.float64)
    cnt = PartCounts()
    rc = lib.dgswem_part_sizes(C.byref(m.s), _ptr(part, C.c_int32), int(n_parts), int(rank), C.byref(cnt))
    if rc != DGSWEM_OK:
        raise DgswemError(rc, "dgswem_part_sizes")
    xy = np.empty((cnt.n_nodes, 2))
    tri = np.empty((cnt.n_elems, 3), np.int32)
    be = np.empty((cnt.n_bedges, 2), np.int32)
    bt = np.empty(cnt.n_bedges, np.int32)
    sub_hb = np.empty(cnt.n_nodes)
    eg = np.empty(cnt.n_elems, np.int32)
    ec = np.empty(cnt.n_elems, np.int32)
    ng = np.empty(cnt.n_nodes, np.int32)
    peer = np.empty(max(cnt.n_peers, 1), np.int32)
    sc = np.empty(max(cnt.n_peers, 1), np.int32)
    rcnt = np.empty(max(cnt.n_peers, 1), np.int32)
    se = np.empty(max(cnt.n_send, 1), np.int32)
    re = np.empty(max(cnt.n_recv, 1), np.int32)
    i32 = C.c_int32
    out = PartOut(_ptr(xy), _ptr(tri, i32), _ptr(be, i32), _ptr(bt, i32), _ptr(sub_hb), _ptr(eg, i32), _ptr(ec, i32),
                  _ptr(ng, i32), _ptr(peer, i32), _ptr(sc, i32), _ptr(rcnt, i32), _ptr(se, i32), _ptr(re, i32))
    rc = lib.dgswem_part_build(C.byref(m.s), _ptr(hb), _ptr(part, C.c_int32), int(n_parts), int(rank), C.byref(out))
    if rc != DGSWEM_OK:
        raise DgswemError(rc, "dgswem_part_build")
    peers = [int(x) for x in peer[:cnt.n_peers]]
    send, recv, a, b = [], [], 0, 0
    for k in range(cnt.n_peers):
        send.append(se[a:a + sc[k]].copy())
        recv.append(re[b:b + rcnt[k]].copy())
        a += sc[k]
        b += rcnt[k]
    return Part(SubMesh(xy, tri, be, bt), sub_hb, eg, ec, ng, peers, send, recv)


class PartModel(Model):
    """One part of a partitioned model (dgswem_create_part + dgswem_attach + dgswem_halo_attach).

    The packed send / receive buffers are torch tensors on the device (float64, one record of
    3 ndof + 1 values per listed element).  A stage is stage_compute(), the delivery of the peers'
    records into recv_buf, then stage_finish().  The delivery must be ordered on the context's
    stream: pass an explicit torch stream (torch's default stream reaches the library as NULL,
    for which the library creates a private non-blocking stream) and enqueue the copies or NCCL
    calls on it."""

    def __init__(self, part: Part, params: dict, init_nodal=None, init_modal=None, t0=0.0, variant=0, block=0,
                 reorder=0, stream=None):
        _Handle.__init__(self)
        mesh = part.mesh
        m = _MeshArrays(mesh)
        hb = np.ascontiguousarray(part.bathy, np.float64)
        self.prm = make_params(params)
        nodal = None if init_nodal is None else np.ascontiguousarray(init_nodal, np.float64)
        modal = None if init_modal is None else np.ascontiguousarray(init_modal, np.float64)
        ini = Init(_ptr(modal), _ptr(nodal), float(t0))
        tun = Tuning(int(variant), int(block), int(reorder), 0)
        self._cls = np.ascontiguousarray(part.elem_class, np.int32)
        self._se = part.send_elems
        self._re = part.recv_elems
        spec = PartSpec(_ptr(self._cls, C.c_int32), len(self._se), _ptr(self._se, C.c_int32), len(self._re),
                        _ptr(self._re, C.c_int32))
        rc = self.lib.dgswem_create_part(C.byref(m.s), _ptr(hb), C.byref(self.prm), C.byref(ini), C.byref(tun),
                                         C.byref(spec), C.byref(self.h))
        if rc != DGSWEM_OK:
            raise DgswemError(rc, "dgswem_create_part")
        self.ne = mesh.n_elems
        self.nn = mesh.n_nodes
        self.nd = (params["p"] + 1) * (params["p"] + 2) // 2
        self.part = part
        self._attach(stream)
        torch = _torch_cuda()
        sb, rb = C.c_size_t(), C.c_size_t()
        self._check(self.lib.dgswem_halo_sizes(self.h, C.byref(sb), C.byref(rb)))
        rec = 3 * self.nd + 1
        self.send_buf = torch.zeros(max(sb.value // 8, 1), dtype=torch.float64, device="cuda")
        self.recv_buf = torch.zeros(max(rb.value // 8, 1), dtype=torch.float64, device="cuda")
        self.record = rec
        self._check(self.lib.dgswem_halo_attach(self.h, _vp(self.send_buf.data_ptr()), _vp(self.recv_buf.data_ptr())))

    def stage_compute(self):
        self._check(self.lib.dgswem_stage_compute(self.h))

    def stage_finish(self):
        self._check(self.lib.dgswem_stage_finish(self.h))
