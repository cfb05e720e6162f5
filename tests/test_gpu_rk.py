"""SSP Runge-Kutta family on the GPU (the paper's DG-optimised SSPRK(s,q) row): every scheme of the
two-register Shu-Osher form, named or given as a coefficient table, matches the oracle to 1e-12
relative L2, with wetting/drying, limiter, tide and a moving storm (stage times)."""
import numpy as np
import pytest

import oracle
from paper_2508_21208_gb300 import Ensemble, Model, synth
from paper_2508_21208_gb300.dgswem import ENSEMBLE_PERSISTENT, VARIANT_SPLIT, VARIANT_TILED

pytestmark = pytest.mark.gpu

SSP33_TABLE = [0.0, 1.0, 1.0, 0.75, 0.25, 0.25, 1.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0]
SCHEMES = [synth.RK_SSP33, synth.RK_SSP32, synth.RK_SSP42, synth.RK_SSP52, synth.RK_SSP43, "custom"]


def with_scheme(prm, scheme):
    prm = dict(prm)
    if scheme == "custom":
        prm.update(rk_scheme=synth.RK_CUSTOM, rk_stages=3, rk_coeffs=SSP33_TABLE)
    else:
        prm["rk_scheme"] = scheme
    return prm


def rel(a, b):
    return max(np.linalg.norm(a[v] - b[v]) / max(np.linalg.norm(b[v]), 1e-300) for v in range(3))


@pytest.mark.parametrize("variant", [VARIANT_SPLIT, VARIANT_TILED])
@pytest.mark.parametrize("scheme", SCHEMES)
def test_shelf_parity(scheme, variant):
    c = synth.config2(n=32)
    prm = with_scheme(c.params, scheme)
    g = Model(c.mesh, c.bathy, prm, init_nodal=c.init_nodal, variant=variant, block=128)
    o = oracle.Oracle(c.mesh, c.bathy, prm, init_nodal=c.init_nodal, omp=True)
    g.step(60)
    o.step(60)
    assert rel(g.state(), o.state()) <= 1e-12
    assert np.array_equal(g.flags(), o.flags())


@pytest.mark.parametrize("scheme", [synth.RK_SSP43, synth.RK_SSP52])
def test_storm_stage_times(scheme):
    c = synth.config3(n=32)
    prm = with_scheme(c.params, scheme)
    g = Model(c.mesh, c.bathy, prm, init_nodal=c.init_nodal, variant=VARIANT_SPLIT, block=128)
    o = oracle.Oracle(c.mesh, c.bathy, prm, init_nodal=c.init_nodal, omp=True)
    g.step(40)
    o.step(40)
    assert rel(g.state(), o.state()) <= 1e-12


def test_ensemble_three_register_scheme_equals_single_runs():
    meshes, bathys, members = synth.ensemble(members_per_mesh=1, mesh_n=(20, 28), precision=synth.FP32_MIXED)
    for _, p, _ in members:
        p.update(track_x0=150e3, rmax_m=60e3, rk_scheme=synth.RK_SSP43)
    ens = Ensemble(meshes, bathys, members, block=64, mode=ENSEMBLE_PERSISTENT)
    ens.step(12)
    for i, (mi, prm, _) in enumerate(members):
        single = Model(meshes[mi], bathys[mi], prm, variant=VARIANT_TILED, block=64)
        single.step(12)
        assert np.array_equal(ens.state(i), single.state())
