"""Rain source and river inflow boundary (Eq. SWE: R and Gamma_river) on the GPU: parity with the
oracle, and the exact water-volume budget through dgswem_mass."""
import numpy as np
import pytest

import oracle
from paper_2508_21208_gb300 import Model, synth
from paper_2508_21208_gb300.dgswem import VARIANT_FUSED, VARIANT_SPLIT, VARIANT_TILED

pytestmark = pytest.mark.gpu


def case():
    mesh = synth.grid_mesh(24, 16, 20e3, 10e3, 5, jitter=0.15, river_sides=("top",), open_sides=("left",))
    x = mesh.xy[:, 0]
    hb = 8.0 - 6.0 * x / 20e3 + 0.5 * np.sin(mesh.xy[:, 1] / 2e3)   # 1.5 .. 8.5 m
    prm = synth.default_params(rain_rate=2e-5, river_q=0.3, cf=0.0025, friction=synth.FRICTION_QUADRATIC,
                               limiter=1, h0=0.01, tide_amp=0.3, tide_period=44714.0)
    init = np.zeros((3, mesh.n_nodes))
    return mesh, hb, prm, init


def rel(a, b):
    return max(np.linalg.norm(a[v] - b[v]) / max(np.linalg.norm(b[v]), 1e-300) for v in range(3))


@pytest.mark.parametrize("flux", [synth.FLUX_LLF, synth.FLUX_ROE])
@pytest.mark.parametrize("variant", [VARIANT_SPLIT, VARIANT_FUSED, VARIANT_TILED])
def test_rain_river_parity(variant, flux):
    mesh, hb, prm, init = case()
    prm["flux"] = flux
    g = Model(mesh, hb, prm, init_nodal=init, variant=variant, block=128)
    o = oracle.Oracle(mesh, hb, prm, init_nodal=init)
    g.step(150)
    o.step(150)
    assert rel(g.state(), o.state()) <= 1e-12
    assert np.array_equal(g.flags(), o.flags())


def test_river_and_rain_volume_budget():
    mesh, hb, prm, init = case()
    prm["tide_amp"] = 0.0
    mesh.bedge_type[mesh.bedge_type == synth.BC_OPEN] = synth.BC_LAND  # closed but for the river
    g = Model(mesh, hb, prm, init_nodal=init)
    dt = g.dt
    _, v0 = g.mass()
    g.step(200)
    _, v1 = g.mass()
    expect = (prm["rain_rate"] * 20e3 * 10e3 + prm["river_q"] * 20e3) * 200 * dt
    assert (v1 - v0) == pytest.approx(expect, rel=1e-11)
