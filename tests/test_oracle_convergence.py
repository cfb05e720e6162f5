"""p+1 convergence of the oracle's whole discretisation on a manufactured smooth solution.

The exact solution w* is smooth; its residual S = dw*/dt + div F(w*) - s(w*) (Eq. SWE, written
out by sympy here) is added as a source, boundary ghosts take w*, and the limiter and wet/dry
are off.  A correct DG discretisation of degree p converges in L2 at rate p+1 (Cockburn & Shu).
"""
import math

import numpy as np
import pytest
import sympy as sp

import oracle
from paper_2508_21208_gb300 import synth

G = 1.0
CF = 0.01
LAT = 30.0


def _exact():
    x, y, t = sp.symbols("x y t")
    hb = 1 + sp.Rational(1, 5) * x + sp.Rational(1, 10) * y
    z = sp.Rational(1, 20) * sp.sin(2 * sp.pi * x + t) * sp.sin(2 * sp.pi * y)
    qx = sp.Rational(1, 20) * (sp.Rational(3, 2) + sp.cos(sp.pi * x) * sp.sin(sp.pi * y) * sp.sin(t + 1))
    qy = sp.Rational(1, 20) * sp.sin(sp.pi * x) * sp.cos(sp.pi * y) * sp.cos(t)
    H = z + hb
    P = G / 2 * (H ** 2 - hb ** 2)
    f = 2 * 7.2921e-5 * math.sin(math.radians(LAT))
    tau = CF * sp.sqrt(qx ** 2 + qy ** 2) / H ** 2
    # conservative form dw/dt + div F(w) = s(w) + S (Eq. SWE); S is the manufactured source
    S0 = sp.diff(z, t) + sp.diff(qx, x) + sp.diff(qy, y)
    S1 = (sp.diff(qx, t) + sp.diff(qx * qx / H + P, x) + sp.diff(qx * qy / H, y)
          - (G * z * sp.diff(hb, x) - tau * qx + f * qy))
    S2 = (sp.diff(qy, t) + sp.diff(qx * qy / H, x) + sp.diff(qy * qy / H + P, y)
          - (G * z * sp.diff(hb, y) - tau * qy - f * qx))
    W = sp.lambdify((t, x, y), [z, qx, qy], "numpy")
    S = sp.lambdify((t, x, y), [S0, S1, S2], "numpy")
    HB = sp.lambdify((x, y), hb, "numpy")

    def wfun(tt, xy):
        return np.stack([np.broadcast_to(v, xy[:, 0].shape) for v in W(tt, xy[:, 0], xy[:, 1])], 1)

    def sfun(tt, xy):
        return np.stack([np.broadcast_to(v, xy[:, 0].shape) for v in S(tt, xy[:, 0], xy[:, 1])], 1)

    return wfun, sfun, HB


WF, SF, HBF = _exact()


def _error(p, n, T=0.2, flux=0):
    mesh = synth.grid_mesh(n, n, 1.0, 1.0, 11)
    hb = HBF(mesh.xy[:, 0], mesh.xy[:, 1])
    h = 1.0 / n
    dt = 0.08 * h if p == 1 else 0.04 * h * math.sqrt(4.0 / n)
    nsteps = int(math.ceil(T / dt))
    dt = T / nsteps
    prm = synth.default_params(p=p, g=G, dt=dt, friction=synth.FRICTION_QUADRATIC, cf=CF,
                               coriolis=1, coriolis_lat_deg=LAT, flux=flux)
    o = oracle.Oracle(mesh, hb, prm)
    o.project(WF, 0.0)
    o.set_mms(SF, WF)
    o.step(nsteps)
    return o.l2err(WF, T)


@pytest.mark.parametrize("flux", [synth.FLUX_LLF, synth.FLUX_ROE])
@pytest.mark.parametrize("p", [1, 2])
def test_convergence_rate(p, flux):
    ns = [4, 8, 16, 32]
    errs = np.array([_error(p, n, flux=flux) for n in ns])
    rates = np.log2(errs[:-1] / errs[1:])
    # the finest two refinements must show the asymptotic rate p+1 in every variable
    assert np.all(rates[-1] > p + 1 - 0.25), (errs, rates)
    assert np.all(rates[-2] > p + 1 - 0.4), (errs, rates)
