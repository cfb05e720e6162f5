"""Pins of the oracle's SSP Runge-Kutta family (Sec. 2.2: Shu-Osher SSPRK, and the paper's
DG-optimised SSPRK(s,q) family) against theory that does not use its coefficient tables.

A uniform state with zero-gradient (transmissive) boundary ghosts has a vanishing spatial
operator, so it evolves by the time integrator alone:
- a linear source (Coriolis rotation) multiplies the state each step by the scheme's stability
  polynomial R(h J): SSP(2,2) 1 + z + z^2/2; SSP(3,3) 1 + z + z^2/2 + z^3/6;
  SSP(s,2) (s-1)/s (1 + z/(s-1))^s + 1/s; SSP(4,3) 1 + z + z^2/2 + z^3/6 + z^4/48;
- a time-dependent source makes the error decay at the scheme's order, which also pins the stage
  times (a wrong stage time drops the order to 1).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2508_21208_gb300 import synth

SCHEMES = {
    synth.RK_SSP22: (2, lambda z: 1 + z + z ** 2 / 2),
    synth.RK_SSP33: (3, lambda z: 1 + z + z ** 2 / 2 + z ** 3 / 6),
    synth.RK_SSP32: (2, lambda z: 2 / 3 * (1 + z / 2) ** 3 + 1 / 3),
    synth.RK_SSP42: (2, lambda z: 3 / 4 * (1 + z / 3) ** 4 + 1 / 4),
    synth.RK_SSP52: (2, lambda z: 4 / 5 * (1 + z / 4) ** 5 + 1 / 5),
    synth.RK_SSP43: (3, lambda z: 1 + z + z ** 2 / 2 + z ** 3 / 6 + z ** 4 / 48),
}


def matpoly(R, M):
    w, V = np.linalg.eig(M)
    return np.real(V @ np.diag([R(x) for x in w]) @ np.linalg.inv(V))


def uniform_model(prm, q0):
    mesh = synth.grid_mesh(4, 4, 40e3, 40e3, 9)
    hb = np.full(mesh.n_nodes, 10.0)
    init = np.zeros((3, mesh.n_nodes))
    init[1], init[2] = q0
    o = oracle.Oracle(mesh, hb, prm, init_nodal=init)
    o.set_transmissive(True)
    return o


@pytest.mark.parametrize("scheme", list(SCHEMES))
def test_coriolis_step_is_stability_polynomial(scheme):
    lat, dt, n = 35.0, 60.0, 20
    f = 2 * 7.2921e-5 * math.sin(math.radians(lat))
    J = f * dt * np.array([[0.0, 1.0], [-1.0, 0.0]])  # q' = f (q_y, -q_x)
    A = matpoly(SCHEMES[scheme][1], J)
    q0 = np.array([0.7, 0.2])
    expect = np.linalg.matrix_power(A, n) @ q0
    o = uniform_model(synth.default_params(coriolis=1, coriolis_lat_deg=lat, dt=dt, rk_scheme=scheme), q0)
    o.step(n)
    u = o.state()
    assert np.allclose(u[1, 0], expect[0], rtol=1e-13, atol=0)
    assert np.allclose(u[2, 0], expect[1], rtol=1e-13, atol=0)
    assert np.abs(u[:, 1:]).max() < 1e-14 and np.abs(u[0]).max() < 1e-14


@pytest.mark.parametrize("scheme", list(SCHEMES))
def test_time_dependent_source_converges_at_scheme_order(scheme):
    order = SCHEMES[scheme][0]
    T, w = 2000.0, 2 * math.pi / 3000.0
    errs = []
    for n in (10, 20, 40):
        o = uniform_model(synth.default_params(dt=T / n, rk_scheme=scheme), (0.0, 0.0))
        # q_x' = cos(w t): exact q_x(T) = sin(w T) / w
        o.set_mms(lambda t, xy: np.tile([0.0, math.cos(w * t), 0.0], (len(xy), 1)),
                  lambda t, xy: np.zeros((len(xy), 3)))
        o.set_transmissive(True)
        o.step(n)
        errs.append(abs(o.state()[1, 0].mean() - math.sin(w * T) / w))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > order - 0.2), (errs, rates)


def test_custom_table_equals_named_scheme():
    q0 = (0.5, -0.3)
    named = uniform_model(synth.default_params(coriolis=1, coriolis_lat_deg=20.0, dt=100.0,
                                               rk_scheme=synth.RK_SSP33), q0)
    coeffs = [0.0, 1.0, 1.0, 0.75, 0.25, 0.25, 1.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0]
    custom = uniform_model(synth.default_params(coriolis=1, coriolis_lat_deg=20.0, dt=100.0,
                                                rk_scheme=synth.RK_CUSTOM, rk_stages=3, rk_coeffs=coeffs), q0)
    named.step(15)
    custom.step(15)
    assert np.array_equal(named.state(), custom.state())


def test_invalid_custom_table_rejected():
    prm = synth.default_params(rk_scheme=synth.RK_CUSTOM, rk_stages=1, rk_coeffs=[0.0, 1.0, 1.0])
    c = synth.config1(n=4)
    with pytest.raises(ValueError):
        oracle.Oracle(c.mesh, c.bathy, prm, init_nodal=c.init_nodal)
