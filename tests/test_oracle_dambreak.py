"""Pin of the oracle against the exact solution of the wet-bed dam break (Stoker 1957), a
closed form the oracle's arithmetic does not use.

The 1D Riemann problem of Eq. SWE with flat bed, depth h_l left and h_r right of x0 at rest,
consists of a left rarefaction and a right shock around a plateau (h_m, u_m):
  rarefaction: u_m = 2 (sqrt(g h_l) - sqrt(g h_m));
  shock (Rankine-Hugoniot of mass and momentum): u_m = (h_m - h_r) sqrt(g (h_m + h_r) / (2 h_m h_r)),
  speed S = h_m u_m / (h_m - h_r);
  inside the fan: h = (2 c_l - xi)^2 / (9 g), u = 2 (c_l + xi) / 3 with xi = (x - x0) / t.
A long channel with walls on its long sides carries it unchanged in 2D. A wrong pressure factor,
flux sign, stage combination or gather would move the plateau, the shock or the fan head.
"""
import math

import numpy as np
import pytest
from scipy.optimize import brentq

import oracle
from paper_2508_21208_gb300 import synth

G = 9.81
HL, HR = 15.0, 10.0
X0, LX, LY = 10e3, 20e3, 200.0
T_END = 400.0


def plateau():
    def f(hm):
        return 2.0 * (math.sqrt(G * HL) - math.sqrt(G * hm)) - (hm - HR) * math.sqrt(G * (hm + HR) / (2 * hm * HR))
    hm = brentq(f, HR * (1 + 1e-12), HL, xtol=1e-14)
    um = 2.0 * (math.sqrt(G * HL) - math.sqrt(G * hm))
    return hm, um, hm * um / (hm - HR)


def exact_depth(x, t):
    hm, um, S = plateau()
    cl, cm = math.sqrt(G * HL), math.sqrt(G * hm)
    xi = (x - X0) / t
    h = np.where(xi < -cl, HL, np.where(xi < um - cm, (2 * cl - xi) ** 2 / (9 * G), np.where(xi < S, hm, HR)))
    return h


def run(nx, flux):
    mesh = synth.grid_mesh(nx, 2, LX, LY, 3)
    hb = np.full(mesh.n_nodes, HR)
    cx = mesh.xy[mesh.tri].mean(axis=1)[:, 0]
    prm = synth.default_params(limiter=1, flux=flux, cfl=0.25)
    u = np.zeros((3, 3, mesh.n_elems))
    u[0, 0] = np.where(cx < X0, HL - HR, 0.0)
    o = oracle.Oracle(mesh, hb, prm, init_modal=u)
    dt = o.dt
    steps = int(round(T_END / dt))
    prm["dt"] = T_END / steps  # land exactly on T_END
    o = oracle.Oracle(mesh, hb, prm, init_modal=u)
    o.step(steps)
    return cx, o.state()


@pytest.mark.parametrize("flux", [synth.FLUX_LLF, synth.FLUX_ROE])
def test_dam_break_matches_stoker(flux):
    hm, um, S = plateau()
    errs = []
    for nx in (200, 400):
        cx, u = run(nx, flux)
        h = u[0, 0] + HR
        dx = LX / nx
        he = exact_depth(cx, T_END)
        errs.append(np.mean(np.abs(h - he)))
        # plateau depth and velocity, away from the fan tail and the shock (whose post-shock
        # wiggle spans a few cells, most with the less dissipative Roe flux)
        xm0, xm1 = X0 + (um - math.sqrt(G * hm)) * T_END + 10 * dx, X0 + S * T_END - 10 * dx
        sel = (cx > xm0) & (cx < xm1)
        assert sel.sum() > 10
        assert np.abs(h[sel] - hm).max() < 0.01 * (hm - HR)
        assert np.abs(u[1, 0][sel] / h[sel] - um).max() < 0.02 * um
        # the shock: first element right of the plateau whose depth is below the mid level
        mid = 0.5 * (hm + HR)
        right = np.where((cx > X0) & (h < mid))[0]
        xs = cx[right].min()
        assert abs(xs - (X0 + S * T_END)) < 3 * dx
        # the fan head has left at -c_l t: undisturbed water ahead of it (beyond the few cells
        # of numerical diffusion), drawn-down water behind
        head = X0 - math.sqrt(G * HL) * T_END
        assert np.abs(h[cx < head - 20 * dx] - HL).max() < 1e-4
        assert h[(cx > head + 10 * dx) & (cx < X0 - 10 * dx)].max() < HL - 0.1
    # first-order convergence in L1 at discontinuities: halving dx cuts the mean error clearly
    assert errs[1] < 0.75 * errs[0], errs
