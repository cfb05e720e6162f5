"""Degenerate and ragged inputs on the GPU against the oracle: a single triangle, meshes smaller than
one tile or warp, a fully dry domain, and zero steps."""
import numpy as np
import pytest

import oracle
from paper_2508_21208_gb300 import Model, synth
from paper_2508_21208_gb300.dgswem import VARIANT_FUSED, VARIANT_SPLIT, VARIANT_TILED

pytestmark = pytest.mark.gpu

VARIANTS = [VARIANT_SPLIT, VARIANT_FUSED, VARIANT_TILED]


def rel(a, b):
    return max(np.linalg.norm(a[v] - b[v]) / max(np.linalg.norm(b[v]), 1e-300) for v in range(3))


def hump_modal(mesh, p=1):
    """A seeded rough modal state over 10 m of water (not from the GPU)."""
    nd = 3 if p == 1 else 6
    rng = np.random.default_rng(5)
    u = np.zeros((3, nd, mesh.n_elems))
    u[0] = 0.05 * rng.standard_normal((nd, mesh.n_elems))
    u[1:] = 0.2 * rng.standard_normal((2, nd, mesh.n_elems))
    return u


@pytest.mark.parametrize("variant", VARIANTS)
def test_single_triangle(variant):
    xy = np.array([[0.0, 0.0], [1000.0, 0.0], [300.0, 900.0]])
    mesh = synth.Mesh(xy, np.array([[0, 1, 2]], np.int32), np.array([[0, 1], [1, 2], [2, 0]], np.int32),
                      np.zeros(3, np.int32))
    hb = np.array([10.0, 12.0, 9.0])
    prm = synth.default_params(friction=synth.FRICTION_QUADRATIC, cf=0.0025, limiter=1)
    u = hump_modal(mesh)
    g = Model(mesh, hb, prm, init_modal=u, variant=variant, block=64)
    o = oracle.Oracle(mesh, hb, prm, init_modal=u)
    g.step(20)
    o.step(20)
    a, b = g.state(), o.state()
    # walls all round: the momentum decays by orders of magnitude, so differences are measured
    # against the scale the run started from
    for v in range(3):
        scale = max(np.linalg.norm(b[v]), np.linalg.norm(u[v]))
        assert np.linalg.norm(a[v] - b[v]) <= 1e-12 * scale
    assert g.mass()[1] == pytest.approx(o.mass()[1], rel=1e-15)


@pytest.mark.parametrize("block", [64, 256])
@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("n", [1, 3, 5])
def test_meshes_smaller_than_a_tile(n, variant, block):
    """2, 18 and 50 elements: fewer than one warp or one tile, ragged everywhere."""
    mesh = synth.grid_mesh(n, n, 5e3, 5e3, 11, jitter=0.1 if n > 1 else 0.0, open_sides=("left",))
    hb = 8.0 + 0.3 * mesh.xy[:, 0] / 5e3
    prm = synth.default_params(friction=synth.FRICTION_QUADRATIC, cf=0.0025, limiter=1, h0=0.01, tide_amp=0.2,
                               tide_period=600.0)
    u = hump_modal(mesh)
    g = Model(mesh, hb, prm, init_modal=u, variant=variant, block=block)
    o = oracle.Oracle(mesh, hb, prm, init_modal=u)
    g.step(60)
    o.step(60)
    assert rel(g.state(), o.state()) <= 1e-12
    assert np.array_equal(g.flags(), o.flags())


@pytest.mark.parametrize("variant", VARIANTS)
def test_fully_dry_domain_stays_at_rest(variant):
    """Land above the datum everywhere, water at h0: every element dry; nothing moves."""
    mesh = synth.grid_mesh(6, 4, 3e3, 2e3, 4)
    hb = -1.0 - 0.5 * mesh.xy[:, 0] / 3e3
    prm = synth.default_params(h0=0.01, limiter=1, friction=synth.FRICTION_QUADRATIC, cf=0.0025)
    init = np.zeros((3, mesh.n_nodes))
    init[0] = 0.01 - hb
    g = Model(mesh, hb, prm, init_nodal=init, variant=variant, block=64)
    o = oracle.Oracle(mesh, hb, prm, init_nodal=init)
    assert np.all(g.flags() == 2) and np.array_equal(g.flags(), o.flags())
    u0 = g.state()
    g.step(50)
    o.step(50)
    u = g.state()
    assert np.all(g.flags() == 2)
    assert np.abs(u[1:]).max() == 0.0
    assert rel(u, o.state()) <= 1e-12
    assert np.abs(u[0] - u0[0]).max() <= 1e-14


def test_zero_steps_leaves_state_unchanged():
    c = synth.config2(n=16)
    g = Model(c.mesh, c.bathy, c.params, init_nodal=c.init_nodal)
    u0 = g.state()
    g.step(0)
    assert np.array_equal(g.state(), u0)
    assert g.info()[2] == 0


def test_blow_up_is_reported_and_sticky():
    """A time step 50x the CFL limit blows the solution up; the kernels' finiteness checks turn
    that into DGSWEM_ENONFINITE at the next synchronising call, and the context stays failed."""
    from paper_2508_21208_gb300.dgswem import DgswemError
    c = synth.config1()
    g0 = Model(c.mesh, c.bathy, c.params, init_nodal=c.init_nodal)
    prm = dict(c.params)
    prm["dt"] = 50.0 * g0.dt
    g = Model(c.mesh, c.bathy, prm, init_nodal=c.init_nodal)
    with pytest.raises(DgswemError) as ei:
        g.step(200)
        g.sync()
    assert ei.value.code == -4
    with pytest.raises(DgswemError):
        g.state()


def test_negative_mean_depth_is_reported():
    """A state whose mean depth is negative cannot be repaired by the wet/dry operator: it
    reports DGSWEM_ENEGDEPTH instead of continuing."""
    from paper_2508_21208_gb300.dgswem import DgswemError
    c = synth.config2(n=16)
    g = Model(c.mesh, c.bathy, c.params, init_nodal=c.init_nodal)
    u = g.state()
    hbm = c.bathy[c.mesh.tri].mean(axis=1)
    u[0, 0, 5] = -hbm[5] - 1.0  # 1 m below the bed
    with pytest.raises(DgswemError) as ei:
        g.set_state(u)  # classifies the state (may already report it)
        g.apply_wetdry()
        g.sync()
    assert ei.value.code == -5
