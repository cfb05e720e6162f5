"""dgswem_mass_noalloc: the mass / volume sums for callers that may not allocate device memory.

Some callers cannot let a library call cudaMalloc: a host model or coupler that owns the GPU's
whole memory budget, or a time-critical loop that cannot afford an allocation's implicit
synchronisation or failure.  This entry point takes only the caller's own device arrays and keeps
its partial sums in a fixed buffer inside the library.  The test checks it against dgswem_mass of
a running model on two calls in a row (the shared buffer must not carry anything over), checks a
ragged element count against an exactly rounded host sum, and checks that null pointers, an empty
input and an oversized input are refused.  The file is named so that pytest collects it last.
"""
import ctypes as C
import math

import numpy as np
import pytest

from paper_2508_21208_gb300 import Model, dgswem, synth

pytestmark = pytest.mark.gpu


def test_noalloc_mass_matches_context_mass_twice():
    import torch

    lib = dgswem.load_library()
    c = synth.config2(n=96)  # 18,432 elements: several partial-sum blocks
    m = Model(c.mesh, c.bathy, c.params, init_nodal=c.init_nodal, variant=1, block=128)
    m.step(15)
    ref_mass, ref_vol = m.mass()
    u = m.state()
    xy, tri = c.mesh.xy, c.mesh.tri
    a = xy[tri[:, 1]] - xy[tri[:, 0]]
    b = xy[tri[:, 2]] - xy[tri[:, 0]]
    area = 0.5 * (a[:, 0] * b[:, 1] - a[:, 1] * b[:, 0])
    hb_mean = c.bathy[tri].mean(axis=1)
    dev = torch.device("cuda")
    z = torch.tensor(u[0, 0], dtype=torch.float64, device=dev)
    ar = torch.tensor(area, dtype=torch.float64, device=dev)
    hb = torch.tensor(hb_mean, dtype=torch.float64, device=dev)
    out = torch.empty(2, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    n = c.mesh.n_elems
    for _ in range(2):
        out.fill_(float("nan"))
        rc = lib.dgswem_mass_noalloc(C.c_void_p(z.data_ptr()), C.c_void_p(ar.data_ptr()),
                                     C.c_void_p(hb.data_ptr()), n, C.c_void_p(out.data_ptr()),
                                     C.c_void_p(stream.cuda_stream))
        assert rc == 0
        stream.synchronize()
        got_mass, got_vol = out.cpu().numpy()
        # same sums in a different element order: equal to rounding of the compensated sums
        assert abs(got_vol - ref_vol) <= 1e-14 * ref_vol
        assert abs(got_mass - ref_mass) <= 1e-14 * ref_vol

    # a ragged count (the last partial-sum block is partly filled, n is no multiple of 2048):
    # the first n - 777 elements, against an exactly rounded host sum of the same terms
    nr = n - 777
    rc = lib.dgswem_mass_noalloc(C.c_void_p(z.data_ptr()), C.c_void_p(ar.data_ptr()),
                                 C.c_void_p(hb.data_ptr()), nr, C.c_void_p(out.data_ptr()),
                                 C.c_void_p(stream.cuda_stream))
    assert rc == 0
    stream.synchronize()
    got_mass, got_vol = out.cpu().numpy()
    zz, aa, hh = u[0, 0, :nr], area[:nr], hb_mean[:nr]
    want_mass = math.fsum(aa * zz)
    want_vol = math.fsum(aa * (zz + hh))
    assert abs(got_mass - want_mass) <= 1e-14 * abs(want_vol)
    assert abs(got_vol - want_vol) <= 1e-14 * abs(want_vol)

    # invalid arguments are refused before any device work
    null = C.c_void_p(0)
    for args in ((null, ar, hb, out), (z, null, hb, out), (z, ar, null, out), (z, ar, hb, null)):
        ptrs = [a if isinstance(a, C.c_void_p) else C.c_void_p(a.data_ptr()) for a in args]
        assert lib.dgswem_mass_noalloc(ptrs[0], ptrs[1], ptrs[2], n, ptrs[3],
                                       C.c_void_p(stream.cuda_stream)) == -1
    assert lib.dgswem_mass_noalloc(C.c_void_p(z.data_ptr()), C.c_void_p(ar.data_ptr()),
                                   C.c_void_p(hb.data_ptr()), 0, C.c_void_p(out.data_ptr()),
                                   C.c_void_p(stream.cuda_stream)) == -1

    too_big = (1 << 26) + 1
    rc = lib.dgswem_mass_noalloc(C.c_void_p(z.data_ptr()), C.c_void_p(ar.data_ptr()),
                                 C.c_void_p(hb.data_ptr()), too_big, C.c_void_p(out.data_ptr()),
                                 C.c_void_p(stream.cuda_stream))
    assert rc == -9
