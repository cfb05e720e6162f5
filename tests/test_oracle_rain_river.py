"""Pins of the rain source and the river inflow boundary (Eq. SWE: R and Gamma_river) by exact
volume budgets: the discrete scheme conserves mass to round-off, so the water volume must change
by exactly R * area * t (rain) and q_in * (river length) * t (river), whatever the flow does."""
import numpy as np
import pytest

import oracle
from paper_2508_21208_gb300 import synth


def basin(n=16, river=False):
    mesh = synth.grid_mesh(n, n, 20e3, 10e3, 5, jitter=0.15, river_sides=("top",) if river else ())
    x = mesh.xy[:, 0]
    hb = 8.0 - 6.0 * x / 20e3 + 0.5 * np.sin(mesh.xy[:, 1] / 2e3)
    return mesh, hb


@pytest.mark.parametrize("flux", [synth.FLUX_LLF, synth.FLUX_ROE])
def test_rain_volume_budget(flux):
    mesh, hb = basin()
    R = 5e-5  # 180 mm/h
    prm = synth.default_params(rain_rate=R, cf=0.0025, friction=synth.FRICTION_QUADRATIC, limiter=1,
                               h0=0.01, dt=10.0, flux=flux)
    o = oracle.Oracle(mesh, hb, prm)
    m0, v0 = o.mass()
    o.step(100)
    m1, v1 = o.mass()
    area = 20e3 * 10e3
    assert (v1 - v0) == pytest.approx(R * area * 1000.0, rel=1e-12)
    assert np.abs(o.state()[1:]).max() > 0  # rain on a sloping bed drives a flow


def test_river_volume_budget_llf():
    mesh, hb = basin(river=True)
    q_in = 0.8  # m^2/s across the 20 km top side
    prm = synth.default_params(river_q=q_in, dt=10.0, limiter=1)
    o = oracle.Oracle(mesh, hb, prm)
    m0, v0 = o.mass()
    o.step(100)
    m1, v1 = o.mass()
    assert (v1 - v0) == pytest.approx(q_in * 20e3 * 1000.0, rel=1e-12)


def test_zero_river_discharge_is_a_wall():
    mesh, hb = basin(river=True)
    mesh_land, _ = basin(river=False)
    prm = synth.default_params(dt=10.0, limiter=1)
    init = np.zeros((3, mesh.n_nodes))
    init[0] = 0.2 * np.exp(-((mesh.xy[:, 0] - 10e3) ** 2 + (mesh.xy[:, 1] - 8e3) ** 2) / 2e3 ** 2)
    a = oracle.Oracle(mesh, hb, prm, init_nodal=init)
    b = oracle.Oracle(mesh_land, hb, prm, init_nodal=init)
    a.step(50)
    b.step(50)
    assert np.array_equal(a.state(), b.state())
