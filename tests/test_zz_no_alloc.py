"""dgswem_mass_noalloc: the mass / volume sums for callers that may not allocate device memory.

Some callers cannot let a library call cudaMalloc: a host model or coupler that owns the GPU's
whole memory budget, or a time-critical loop that cannot afford an allocation's implicit
synchronisation or failure.  This entry point takes only the caller's own device arrays and keeps
its partial sums in a fixed buffer inside the library.  The test checks it against dgswem_mass of
a running model on two calls in a row (the shared buffer must not carry anything over), and that
an oversized input is refused.  The file is named so that pytest collects it last.
"""
import ctypes as C

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

    too_big = (1 << 26) + 1
    rc = lib.dgswem_mass_noalloc(C.c_void_p(z.data_ptr()), C.c_void_p(ar.data_ptr()),
                                 C.c_void_p(hb.data_ptr()), too_big, C.c_void_p(out.data_ptr()),
                                 C.c_void_p(stream.cuda_stream))
    assert rc == -9
