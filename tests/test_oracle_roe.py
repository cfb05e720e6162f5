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


# ------------------------------------------------------------------ no water: H <= 0
def _pressure_only(g, w, hb, nx, ny):
    """F(w).n with zero velocity: (q.n, P n_x, P n_y), P = (g/2) zeta (zeta + 2 h_b)."""
    P = 0.5 * g * w[0] * (w[0] + 2.0 * hb)
    return np.array([w[1] * nx + w[2] * ny, P * nx, P * ny])


@pytest.mark.parametrize("params", [LLF, ROE], ids=["llf", "roe"])
def test_no_water_side_has_zero_velocity(params):
    """Where the total depth is not positive, the velocity q/H and the wave speed are zero: the
    equations divide by H with no rule for H <= 0, and both fluxes take this one.  With both sides
    dry the flux is the mean of the pressure-only fluxes (no dissipation: every wave speed is 0);
    with one dry side the LLF flux takes the wet side's wave speed alone, written out here."""
    g = params["g"]
    rng = np.random.default_rng(5)
    for _ in range(100):
        hb = rng.uniform(0.5, 5.0)
        th = rng.uniform(0, 2 * math.pi)
        nx, ny = math.cos(th), math.sin(th)
        a = np.array([-hb - rng.uniform(0.0, 1.0), rng.normal(), rng.normal()])  # H <= 0
        b = np.array([-hb - rng.uniform(0.1, 1.0), rng.normal(), rng.normal()])  # H < 0
        want = 0.5 * (_pressure_only(g, a, hb, nx, ny) + _pressure_only(g, b, hb, nx, ny))
        assert np.allclose(oracle.numflux(params, a, b, hb, nx, ny), want, rtol=1e-14, atol=1e-13)
    a = np.array([-3.0, 0.0, 0.0])             # exactly no water: H = 0
    b = np.array([-2.5, 1.0, -2.0])            # wet: H = 0.5
    hb, nx, ny = 3.0, 0.6, 0.8
    f = oracle.numflux(params, a, b, hb, nx, ny)
    assert np.all(np.isfinite(f))
    if params is LLF:
        Hb = b[0] + hb
        lam = abs((b[1] * nx + b[2] * ny) / Hb) + math.sqrt(g * Hb)
        qnb = b[1] * nx + b[2] * ny
        Fb = np.array([qnb, b[1] * qnb / Hb, b[2] * qnb / Hb]) + _pressure_only(g, b, hb, nx, ny) * [0, 1, 1]
        want = 0.5 * (_pressure_only(g, a, hb, nx, ny) + Fb) - 0.5 * lam * (b - a)
        assert np.allclose(f, want, rtol=1e-14, atol=1e-13)


def test_no_water_momentum_rhs_does_not_depend_on_momentum():
    """With the total depth negative everywhere (wetting/drying off, no Coriolis), the momentum rows
    of the right-hand side come from the pressure and bed-slope terms only: no advection, no
    friction, no LLF dissipation.  Two different momentum fields must give the same rows; a
    division by H anywhere (area, edge or friction) would make them differ."""
    c = synth.config1(n=6)
    prm = dict(c.params, h0=0.0, coriolis=0, dt=1.0)  # Manning friction on; no CFL step without water
    hb = c.bathy
    rng = np.random.default_rng(3)
    nd = 3
    u = np.zeros((3, nd, c.mesh.n_elems))
    tri = c.mesh.tri
    # zeta at the vertices 0.2 to 1.2 m below the bed: H < 0 at every point of every element
    for e in range(c.mesh.n_elems):
        zv = -hb[tri[e]] - rng.uniform(0.2, 1.2, 3)
        u[0, :, e] = [zv.mean(), 0.5 * (zv[1] - zv[0]), (2.0 * zv[2] - zv[0] - zv[1]) / 6.0]
    rows = []
    for seed in (1, 2):
        v = u.copy()
        v[1:] = np.random.default_rng(seed).normal(size=(2, nd, c.mesh.n_elems))
        o = oracle.Oracle(c.mesh, c.bathy, prm, init_modal=v)
        o.set_state(v)
        r = o.rhs(0.0)
        assert np.all(np.isfinite(r))
        rows.append(r[1:])
    assert np.array_equal(rows[0], rows[1])
