"""CPU checks of the C-ABI library: it loads, exports every declared entry point, and rejects
invalid meshes and parameters on the host (dgswem_create does no device work)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2508_21208_gb300 import dgswem, synth
from paper_2508_21208_gb300.build import build_library

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build_library()
    return dgswem.load_library()


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "dgswem.h")).read()
    return sorted(set(re.findall(r"DGSWEM_API\s+[\w\s\*]*?\b(dgswem_\w+)\s*\(", txt)))


def test_exports_every_declared_symbol(lib):
    names = declared_symbols()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(s for s, _, _ in dgswem.SIGNATURES) == names


def _create(mesh, bathy, params, tuning=None):
    lib = dgswem.load_library()
    m = dgswem._MeshArrays(mesh)
    hb = np.ascontiguousarray(bathy, np.float64)
    prm = dgswem.make_params(params)
    h = C.c_void_p()
    tun = tuning or dgswem.Tuning(0, 0, 0, 0)
    rc = lib.dgswem_create(C.byref(m.s), dgswem._ptr(hb), C.byref(prm), None, C.byref(tun), C.byref(h))
    return rc, h


def test_create_and_workspace_size(lib):
    c = synth.config1(n=8)
    rc, h = _create(c.mesh, c.bathy, c.params)
    assert rc == 0 and h
    n = C.c_size_t()
    assert lib.dgswem_workspace_size(h, C.byref(n)) == 0
    assert n.value > 128 * 8 * 2 * 9 * 2
    # state calls before attach are rejected, not crashed
    assert lib.dgswem_step(h, 1) == -8
    lib.dgswem_destroy(h)


@pytest.mark.parametrize("bad", ["clockwise", "index", "nonmanifold", "bedge"])
def test_invalid_mesh_rejected(lib, bad):
    c = synth.config1(n=4)
    m = c.mesh
    tri, bedge = m.tri.copy(), m.bedge.copy()
    if bad == "clockwise":
        tri[3] = tri[3][::-1]
    elif bad == "index":
        tri[2, 1] = m.n_nodes + 5
    elif bad == "nonmanifold":
        tri = np.concatenate([tri, tri[:1]])
    elif bad == "bedge":
        bedge[0] = [0, m.n_nodes - 1]
    mesh = synth.Mesh(m.xy, tri.astype(np.int32), bedge.astype(np.int32), m.bedge_type)
    rc, h = _create(mesh, c.bathy, c.params)
    assert rc == -2 and not h


@pytest.mark.parametrize("key,val", [("p", 3), ("g", -1.0), ("h0", -0.1), ("friction", 7), ("precision", 5)])
def test_invalid_params_rejected(lib, key, val):
    c = synth.config1(n=4)
    prm = dict(c.params)
    prm[key] = val
    rc, h = _create(c.mesh, c.bathy, prm)
    assert rc == -1 and not h


def test_nan_bathymetry_rejected(lib):
    c = synth.config1(n=4)
    hb = c.bathy.copy()
    hb[3] = np.nan
    rc, h = _create(c.mesh, hb, c.params)
    assert rc == -1


@pytest.mark.parametrize("key,val", [("flux", 2), ("rk_scheme", 9), ("rain_rate", float("nan")),
                                     ("river_q", float("inf")), ("dt", -1.0), ("tide_phase", float("nan")),
                                     ("cf", float("inf"))])
def test_more_invalid_params_rejected(lib, key, val):
    c = synth.config1(n=4)
    prm = dict(c.params)
    prm[key] = val
    rc, h = _create(c.mesh, c.bathy, prm)
    assert rc == -1 and not h


def test_custom_rk_table_with_nan_rejected(lib):
    c = synth.config1(n=4)
    prm = dict(c.params, rk_scheme=synth.RK_CUSTOM, rk_stages=2, rk_coeffs=[0, 1, 1, 0.5, 0.5, float("nan")])
    rc, h = _create(c.mesh, c.bathy, prm)
    assert rc == -1 and not h


def _one_triangle(p2):
    xy = np.array([[0.0, 0.0], [1000.0, 0.0], p2])
    return synth.Mesh(xy, np.array([[0, 1, 2]], np.int32), np.array([[0, 1], [1, 2], [2, 0]], np.int32),
                      np.zeros(3, np.int32))


def test_empty_mesh_rejected(lib):
    m = synth.Mesh(np.zeros((0, 2)), np.zeros((0, 3), np.int32), np.zeros((0, 2), np.int32), np.zeros(0, np.int32))
    rc, h = _create(m, np.zeros(0), synth.config1(n=4).params)
    assert rc == -1 and not h


def test_zero_area_triangle_rejected(lib):
    rc, h = _create(_one_triangle([2000.0, 0.0]), np.full(3, 10.0), synth.config1(n=4).params)
    assert rc == -2 and not h


def test_single_triangle_accepted(lib):
    rc, h = _create(_one_triangle([0.0, 1000.0]), np.full(3, 10.0), synth.config1(n=4).params)
    assert rc == 0 and h
    lib.dgswem_destroy(h)


def _ens_create(lib, meshes, bathys, members):
    marr = [dgswem._MeshArrays(m) for m in meshes]
    hbs = [np.ascontiguousarray(b, np.float64) for b in bathys]
    n = len(members)
    mesh_ptrs = (C.POINTER(dgswem.Mesh) * n)()
    hb_ptrs = (C.POINTER(C.c_double) * n)()
    prms = (dgswem.Params * n)()
    inits = (dgswem.Init * n)()
    for i, (mi, prm) in enumerate(members):
        mesh_ptrs[i] = C.pointer(marr[mi].s)
        hb_ptrs[i] = dgswem._ptr(hbs[mi])
        prms[i] = dgswem.make_params(prm)
        inits[i] = dgswem.Init(None, None, 0.0)
    h = C.c_void_p()
    rc = lib.dgswem_ensemble_create(n, mesh_ptrs, hb_ptrs, prms, inits, C.byref(dgswem.Tuning(0, 0, 0, 0)), C.byref(h))
    if rc == 0:
        lib.dgswem_destroy(h)
    return rc


@pytest.mark.parametrize("key,val", [("p", 2), ("precision", synth.FP32_MIXED), ("rk_scheme", synth.RK_SSP33)])
def test_ensemble_members_must_share_degree_precision_and_scheme(lib, key, val):
    c = synth.config1(n=6)
    other = dict(c.params)
    other[key] = val
    assert _ens_create(lib, [c.mesh], [c.bathy], [(0, c.params), (0, dict(c.params))]) == 0
    assert _ens_create(lib, [c.mesh], [c.bathy], [(0, c.params), (0, other)]) == -1


def test_ensemble_step_refuses_a_single_model_context(lib):
    c = synth.config1(n=4)
    rc, h = _create(c.mesh, c.bathy, c.params)
    assert rc == 0
    assert lib.dgswem_ensemble_step(h, 1) == -1
    lib.dgswem_destroy(h)


@pytest.mark.parametrize("kind", ["one byte short", "null"])
def test_attach_with_a_short_workspace_is_enomem(lib, kind):
    """Allocator failure simulated by a size cap: a workspace one byte smaller than
    dgswem_workspace_size (or none) is refused with DGSWEM_ENOMEM, and the error is sticky.  The
    size check comes before any device work, so the (never dereferenced) address below is safe and
    no GPU is needed."""
    c = synth.config1(n=8)
    rc, h = _create(c.mesh, c.bathy, c.params)
    assert rc == 0
    n = C.c_size_t()
    assert lib.dgswem_workspace_size(h, C.byref(n)) == 0
    addr = C.c_void_p(1 << 20) if kind == "one byte short" else C.c_void_p(0)
    assert lib.dgswem_attach(h, addr, n.value - 1, None) == -7
    assert b"workspace" in lib.dgswem_last_error(h)
    assert lib.dgswem_step(h, 1) == -7  # sticky
    lib.dgswem_destroy(h)
