"""The open (tidal) boundary against the linear long-wave solution (§2.1 Gamma_ocean, Alg. 2).

A channel of constant depth D at rest is forced at x = 0 by the tide zeta(0, t) = A sin(w t).
For A << D the shallow water equations are the linear wave equation, and the solution is the
wave travelling in from the boundary, zeta = A sin(w (t - x/c)), q_x = c zeta, c = sqrt(g D),
ahead of which the water is still.  This wave is a fixed point of the boundary treatment
(ghost zeta = tide, ghost q = interior q gives the ghost the interior's state), so the element
means behind its front converge to it at the method's order.
"""
import numpy as np
import pytest

import oracle
from paper_2508_21208_gb300 import synth

G, D, A, PERIOD = 9.81, 10.0, 1e-4, 3600.0
W, C = 2.0 * np.pi / PERIOD, np.sqrt(G * D)
LX, LY, T_END = 80e3, 5e3, 5000.0


def mean_error(nx, flux=0):
    """Mean |zeta_00 - zeta_exact| / A over elements at least 3 cells behind the front."""
    mesh = synth.grid_mesh(nx, max(2, nx // 16), LX, LY, seed=7, jitter=0.2, open_sides=("left",))
    prm = synth.default_params(tide_amp=A, tide_period=PERIOD, flux=flux)
    o = oracle.Oracle(mesh, np.full(mesh.n_nodes, D), prm, init_nodal=np.zeros((3, mesh.n_nodes)))
    steps = int(round(T_END / o.dt))
    o.step(steps)
    t = steps * o.dt
    x = mesh.xy[mesh.tri].mean(axis=1)[:, 0]
    behind = x < C * t - 3.0 * LX / nx
    ze = A * np.sin(W * (t - x / C))  # barycentre value: the element mean to O(h^2)
    u = o.state()
    return (np.abs(u[0, 0] - ze)[behind].mean() / A,
            np.abs(u[1, 0] - C * ze)[behind].mean() / (C * A))


@pytest.mark.parametrize("flux", [0, 1])  # LLF, Roe
def test_tidal_wave_converges_at_second_order(flux):
    e = [mean_error(nx, flux) for nx in (32, 64, 128)]
    z = [a for a, _ in e]
    q = [b for _, b in e]
    assert z[2] < 1e-3 and q[2] < 1e-3          # LLF 6.6e-4 and 7.2e-4 of the amplitude; Roe 4.6e-4
    for k in range(2):                          # measured ratios 3.4 (LLF) and 3.6-3.8 (Roe)
        assert z[k] / z[k + 1] > 2.5 and q[k] / q[k + 1] > 2.5
