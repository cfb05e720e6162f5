"""Pins of the oracle's Roe flux (Sec. 2.2 names LLF or Roe as the numerical flux).

- consistency: Fhat(w, w) = F(w).n, taken from the LLF flux (pinned elsewhere), whose value at
  equal states is F(w).n;
- conservation: Fhat(a, b, n) = -Fhat(b, a, -n);
- the Roe property F(b) - F(a) = A~ (b - a): when every Roe eigenvalue is positive (supersonic flow
  towards the outer state), the flux is exactly the inner physical flux, and with every eigenvalue
  negative exactly the outer one;
- lake at rest, mass conservation with wetting/drying, p+1 convergence.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2508_21208_gb300 import synth

ROE = synth.default_params(flux=synth.FLUX_ROE)
LLF = synth.default_params(flux=synth.FLUX_LLF)


def rand_state(rng, hb, speed):
    z = 0.5 * rng.standard_normal()
    H = z + hb
    ang = rng.uniform(0, 2 * math.pi)
    return np.array([z, H * speed * math.cos(ang), H * speed * math.sin(ang)])


def test_consistency_and_conservation():
    rng = np.random.default_rng(0)
    for _ in range(200):
        hb = rng.uniform(1.0, 50.0)
        a = rand_state(rng, hb, rng.uniform(0, 5))
        b = rand_state(rng, hb, rng.uniform(0, 5))
        th = rng.uniform(0, 2 * math.pi)
        nx, ny = math.cos(th), math.sin(th)
        Fa = oracle.numflux(LLF, a, a, hb, nx, ny)
        assert np.allclose(oracle.numflux(ROE, a, a, hb, nx, ny), Fa, rtol=1e-14, atol=1e-13)
        f1 = oracle.numflux(ROE, a, b, hb, nx, ny)
        f2 = oracle.numflux(ROE, b, a, hb, -nx, -ny)
        assert np.allclose(f1, -f2, rtol=1e-13, atol=1e-12)


@pytest.mark.parametrize("direction", [1.0, -1.0])
def test_supersonic_flux_is_upwind(direction):
    rng = np.random.default_rng(1)
    g = 9.81
    for _ in range(200):
        hb = rng.uniform(0.5, 5.0)
        th = rng.uniform(0, 2 * math.pi)
        nx, ny = math.cos(th), math.sin(th)

        def state():
            z = rng.uniform(-0.2, 0.2)
            H = z + hb
            un = direction * (3.0 + rng.uniform(0, 2)) * math.sqrt(g * H)  # |u.n| > 3 c
            ut = rng.uniform(-1, 1)
            return np.array([z, H * (un * nx - ut * ny), H * (un * ny + ut * nx)])

        a, b = state(), state()
        up = a if direction > 0 else b
        Fup = oracle.numflux(LLF, up, up, hb, nx, ny)
        F = oracle.numflux(ROE, a, b, hb, nx, ny)
        assert np.allclose(F, Fup, rtol=1e-12, atol=1e-10 * np.abs(Fup).max())


def test_lake_at_rest_and_mass_with_roe():
    c = synth.config1(lake=True)
    c.init_nodal[0] = 0.3
    c.params["flux"] = synth.FLUX_ROE
    o = oracle.Oracle(c.mesh, c.bathy, c.params, init_nodal=c.init_nodal)
    o.step(100)
    u = o.state()
    assert np.abs(u[1:]).max() < 1e-11
    c = synth.config2(n=24)
    c.mesh.bedge_type[:] = synth.BC_LAND
    c.params.update(tide_amp=0.0, flux=synth.FLUX_ROE)
    x = c.mesh.xy[:, 0]
    c.init_nodal[0] = np.where(c.bathy > 0, 0.5 * np.exp(-((x - 80e3) / 5e3) ** 2), c.init_nodal[0])
    o = oracle.Oracle(c.mesh, c.bathy, c.params, init_nodal=c.init_nodal)
    m0, v0 = o.mass()
    o.step(200)
    m1, v1 = o.mass()
    assert abs(v1 - v0) <= 1e-14 * v0
    assert np.all(np.isfinite(o.state()))
