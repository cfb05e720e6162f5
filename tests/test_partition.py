"""Domain decomposition (Sec. 5.3) on the CPU: the library's host partitioner and sub-mesh builder,
and a two-rank run of the oracle on the parts with one ghost exchange per Runge-Kutta stage
through torch.distributed (gloo), whose union must equal the single-domain oracle bit for bit.

The partitioned run is exact because each part holds two ghost layers: it updates its own
elements and the first layer with every input the single-domain run uses (states and wet/dry
flags of the elements around them), limits and wets/dries its own elements with the first layer's
means, and then takes the ghost states and flags from their owners.  The sub-mesh keeps the
global element and node order, so every edge keeps its orientation and its flux is evaluated
with the same operands in the same order.
"""
import os
import socket
from collections import deque

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from paper_2508_21208_gb300 import dgswem, synth


def _neighbours(mesh):
    tri = mesh.tri
    seen, nbr = {}, -np.ones((mesh.n_elems, 3), int)
    for e in range(mesh.n_elems):
        for l in range(3):
            k = tuple(sorted((int(tri[e, (l + 1) % 3]), int(tri[e, (l + 2) % 3]))))
            if k in seen:
                f, lf = seen.pop(k)
                nbr[e, l], nbr[f, lf] = f, e
            else:
                seen[k] = (e, l)
    return nbr


def _distances(nbr, own):
    """Face-step distance of every element from the element set `own` (breadth-first)."""
    d = np.full(len(nbr), 99)
    q = deque(np.flatnonzero(own))
    d[own] = 0
    while q:
        e = q.popleft()
        for j in nbr[e]:
            if j >= 0 and d[j] > d[e] + 1:
                d[j] = d[e] + 1
                q.append(j)
    return d


@pytest.mark.parametrize("n_parts", [1, 2, 3, 5, 8])
def test_rcb_balanced_deterministic(n_parts):
    c = synth.config2(n=24)  # 1,152 elements
    part = dgswem.partition_rcb(c.mesh, n_parts)
    counts = np.bincount(part, minlength=n_parts)
    assert counts.sum() == c.mesh.n_elems and counts.min() >= 1
    assert counts.max() - counts.min() <= 1
    assert np.array_equal(part, dgswem.partition_rcb(c.mesh, n_parts))


def test_rcb_parts_are_compact():
    """Bisection along coordinates: two parts of the square-ish shelf split along x."""
    c = synth.config2(n=24)
    part = dgswem.partition_rcb(c.mesh, 2)
    cx = c.mesh.xy[c.mesh.tri].mean(axis=1)[:, 0]
    assert cx[part == 0].max() <= cx[part == 1].min()


@pytest.mark.parametrize("n_parts", [2, 4])
def test_parts_ghost_layers_and_matching_lists(n_parts):
    c = synth.config2(n=16, seed=7)
    mesh = c.mesh
    part = dgswem.partition_rcb(mesh, n_parts)
    nbr = _neighbours(mesh)
    parts = [dgswem.build_part(mesh, c.bathy, part, n_parts, r) for r in range(n_parts)]
    for r, P in enumerate(parts):
        d = _distances(nbr, part == r)
        keep = np.flatnonzero(d <= 2)
        assert np.array_equal(P.elem_global, keep)                 # increasing global order
        assert np.array_equal(P.elem_class, d[keep])               # own, layer 1, layer 2
        assert np.all(np.diff(P.node_global) > 0)
        # the sub-mesh is the global mesh restricted to these elements
        assert np.array_equal(P.node_global[P.mesh.tri], mesh.tri[keep])
        assert np.allclose(P.mesh.xy, mesh.xy[P.node_global]) and np.array_equal(P.bathy, c.bathy[P.node_global])
        # every ghost is received exactly once, from its owner
        recv = np.concatenate(P.recv) if P.recv else np.zeros(0, int)
        assert sorted(recv) == sorted(np.flatnonzero(P.elem_class > 0))
        for q, rl in zip(P.peers, P.recv):
            assert np.all(part[P.elem_global[rl]] == q)
    # r's send group for q and q's receive group for r name the same elements in the same order
    for r, P in enumerate(parts):
        for q, sl in zip(P.peers, P.send):
            Q = parts[q]
            rl = Q.recv[Q.peers.index(r)]
            assert np.array_equal(P.elem_global[sl], Q.elem_global[rl])
            assert np.all(P.elem_class[sl] == 0)


def test_part_keeps_boundary_types():
    c = synth.config2(n=16)  # open boundary at x = 0, land elsewhere
    part = dgswem.partition_rcb(c.mesh, 2)
    for r in range(2):
        P = dgswem.build_part(c.mesh, c.bathy, part, 2, r)
        gb = {tuple(sorted(e)): t for e, t in zip(c.mesh.bedge.tolist(), c.mesh.bedge_type.tolist())}
        for e, t in zip(P.mesh.bedge.tolist(), P.mesh.bedge_type.tolist()):
            assert gb[tuple(sorted(P.node_global[e].tolist()))] == t
    assert dgswem.build_part(c.mesh, c.bathy, part, 2, 0).mesh.bedge_type.tolist().count(synth.BC_OPEN) > 0


# ------------------------------------------------------------------ two ranks, gloo, oracle
def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _case(name):
    if name == "800-triangle hump":
        c = synth.config1(n=20)
        return c, 60
    if name == "shelf at p=2":
        return synth.config2(n=20, p=2), 40  # quadratic modes: 6 per variable in each record
    c = synth.config2(n=48)  # 4,608 elements: tide, dry land, wet/dry, limiter, friction
    return c, 60


def _rank_main(rank, world, port, name, out):
    import torch
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        c, steps = _case(name)
        dt = oracle.Oracle(c.mesh, c.bathy, c.params, init_nodal=c.init_nodal).dt
        prm = dict(c.params, dt=dt)
        part = dgswem.partition_rcb(c.mesh, world)
        P = dgswem.build_part(c.mesh, c.bathy, part, world, rank)
        nodal = None if c.init_nodal is None else c.init_nodal[:, P.node_global]
        o = oracle.Oracle(P.mesh, P.bathy, prm, init_nodal=nodal)
        nd = o.nd
        for _ in range(steps):
            for _ in range(o.stage_count()):
                r = o.stage()
                u, f = o.register(r), o.flags()
                reqs, inbox = [], []
                for q, sl, rl in zip(P.peers, P.send, P.recv):
                    rec = np.concatenate([u[:, :, sl].reshape(3 * nd, -1), f[sl][None, :].astype(np.float64)])
                    reqs.append(dist.isend(torch.from_numpy(np.ascontiguousarray(rec)), q))
                    buf = torch.empty((3 * nd + 1, len(rl)), dtype=torch.float64)
                    reqs.append(dist.irecv(buf, q))
                    inbox.append((rl, buf))
                for rq in reqs:
                    rq.wait()
                for rl, buf in inbox:
                    b = buf.numpy()
                    u[:, :, rl] = b[:3 * nd].reshape(3, nd, -1)
                    f[rl] = b[3 * nd].astype(np.uint8)
                o.set_register(r, u)
                o.set_flags(f)
        own = P.elem_class == 0
        out.put((rank, P.elem_global[own], o.state()[:, :, own], o.flags()[own]))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("name", ["800-triangle hump", "shelf with dry land", "shelf at p=2"])
def test_two_ranks_with_ghost_exchange_equal_single_domain_bitwise(name):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, name, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(2)]
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    c, steps = _case(name)
    ref = oracle.Oracle(c.mesh, c.bathy, c.params, init_nodal=c.init_nodal)
    ref.step(steps)
    u, f = ref.state(), ref.flags()
    got_u, got_f = np.full_like(u, np.nan), np.full(len(f), 255, np.uint8)
    for _, g, s, fl in res:
        got_u[:, :, g] = s
        got_f[g] = fl
    assert not np.isnan(got_u).any()
    assert np.array_equal(got_u, u)          # bit for bit
    assert np.array_equal(got_f, f)
    if name != "800-triangle hump":
        assert (f != 0).any() and (f == 0).any()
