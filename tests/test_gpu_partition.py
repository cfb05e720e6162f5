"""Domain decomposition on the GPU (Sec. 5.3): parts of one model, each a context with two ghost
layers, stepped stage by stage with the library's pack / unpack kernels and the packed records
moved between the parts' device buffers by the caller (here copies on one GPU; NCCL or MPI
between GPUs).  The parts' own elements together must match the single-domain oracle."""
import numpy as np
import pytest

import oracle
from paper_2508_21208_gb300 import dgswem, synth

pytestmark = pytest.mark.gpu

STAGES = {synth.RK_SSP22: 2, synth.RK_SSP33: 3, synth.RK_SSP32: 3, synth.RK_SSP42: 4, synth.RK_SSP52: 5,
          synth.RK_SSP43: 4}


def run_parts(c, n_parts, steps, variant=0, block=0):
    import torch

    ref = oracle.Oracle(c.mesh, c.bathy, dict(c.params, precision=synth.FP64), init_nodal=c.init_nodal)
    prm = dict(c.params, dt=ref.dt)
    part = dgswem.partition_rcb(c.mesh, n_parts)
    parts = [dgswem.build_part(c.mesh, c.bathy, part, n_parts, r) for r in range(n_parts)]
    # every part and every copy on one stream, which orders each part's pack, the copies and the
    # unpacks (with several GPUs: one stream per part, the copies replaced by NCCL send/recv)
    st = torch.cuda.Stream()
    models = [dgswem.PartModel(P, prm, init_nodal=c.init_nodal[:, P.node_global], variant=variant, block=block,
                               stream=st) for P in parts]
    rec = models[0].record
    with torch.cuda.stream(st):
        for _ in range(steps):
            for _ in range(STAGES[c.params["rk_scheme"]]):
                for m in models:
                    m.stage_compute()
                for r, (P, m) in enumerate(zip(parts, models)):
                    off = 0
                    for q, rl in zip(P.peers, P.recv):
                        Q = parts[q]
                        k = Q.peers.index(r)
                        src = sum(len(x) for x in Q.send[:k]) * rec
                        n = len(rl) * rec
                        m.recv_buf[off:off + n].copy_(models[q].send_buf[src:src + n])
                        off += n
                for m in models:
                    m.stage_finish()
    nd = models[0].nd
    u = np.full((3, nd, c.mesh.n_elems), np.nan)
    f = np.full(c.mesh.n_elems, 255, np.uint8)
    mass = 0.0
    for P, m in zip(parts, models):
        own = P.elem_class == 0
        u[:, :, P.elem_global[own]] = m.state()[:, :, own]
        f[P.elem_global[own]] = m.flags()[own]
        mass += m.mass()[0]
    ref.step(steps)
    return u, f, mass, ref


def rel_l2(a, b):
    return np.array([np.linalg.norm(a[v] - b[v]) / max(np.linalg.norm(b[v]), 1e-300) for v in range(3)])


@pytest.mark.parametrize("variant", [dgswem.VARIANT_SPLIT, dgswem.VARIANT_FUSED, dgswem.VARIANT_TILED])
def test_three_parts_shelf_fp64_match_oracle(variant):
    c = synth.config2(n=48)  # tide, dry land, wet/dry, limiter, friction
    u, f, mass, ref = run_parts(c, 3, 100, variant=variant, block=128)
    assert not np.isnan(u).any()
    assert np.all(rel_l2(u, ref.state()) <= 1e-12)
    assert np.array_equal(f, ref.flags())
    m_ref, vol = ref.mass()
    assert abs(mass - m_ref) <= 1e-12 * vol


def test_two_parts_p2_and_four_parts_hump():
    c = synth.config2(n=24, p=2)
    u, f, _, ref = run_parts(c, 2, 60)
    assert np.all(rel_l2(u, ref.state()) <= 1e-12) and np.array_equal(f, ref.flags())
    c = synth.config1(n=20)
    u, f, _, ref = run_parts(c, 4, 100)
    assert np.all(rel_l2(u, ref.state()) <= 1e-12)


def test_two_parts_mixed_form_within_its_bound():
    c = synth.config2(n=48, precision=synth.FP32_MIXED)
    u, f, _, ref = run_parts(c, 2, 100)
    b = ref.state()
    assert np.abs(u[0, 0] - b[0, 0]).max() <= 1e-4 and np.array_equal(f, ref.flags())


def test_part_refuses_whole_steps_and_needs_fixed_dt():
    c = synth.config2(n=16)
    part = dgswem.partition_rcb(c.mesh, 2)
    P = dgswem.build_part(c.mesh, c.bathy, part, 2, 0)
    with pytest.raises(dgswem.DgswemError):  # dt = 0 (CFL): a part needs the global fixed dt
        dgswem.PartModel(P, c.params, init_nodal=c.init_nodal[:, P.node_global])
    m = dgswem.PartModel(P, dict(c.params, dt=0.5), init_nodal=c.init_nodal[:, P.node_global])
    with pytest.raises(dgswem.DgswemError):
        m.step(1)
