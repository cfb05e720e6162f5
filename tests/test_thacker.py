"""Thacker's (1981) planar solution in a parabolic bowl: a closed-form pin of the wetting/drying
treatment with a moving shoreline (the paper's WETDRY kernel and the edge rule, §5.2.3).

In the bowl h_b = D0 (1 - r^2/L^2) the water body keeps the bowl's shape and slides rigidly:
its centre sits at x_c(t) = eta cos(w t), w = sqrt(2 g D0) / L, the velocity is uniform,
u = -eta w sin(w t), and the surface is the plane
    zeta(x, t) = (2 D0 eta / L^2) x cos(w t) - (D0 eta^2 / L^2) cos^2(w t)
wherever the depth zeta + h_b is positive (derived from the inviscid equations: u_t + g zeta_x = 0
and zeta_t + (H u)_x = 0 hold identically).  After half a period the body has moved 2 eta across
the bowl, its shoreline wetting one side and drying the other.  The oracle's element means in the
wet interior must converge to the plane on refinement, without and with rotation (below); on the
GPU the FP64 form must match the oracle through the moving front, and the FP32-mixed form must
track the plane as closely.
"""
import numpy as np
import pytest

import oracle
from paper_2508_21208_gb300 import synth

G, D0, L, ETA, H0 = 9.81, 10.0, 10e3, 1000.0, 0.01
W = np.sqrt(2.0 * G * D0) / L


def exact_zeta(x, t):
    return (2.0 * D0 * ETA / L**2) * x * np.cos(W * t) - (D0 * ETA**2 / L**2) * np.cos(W * t) ** 2


def bowl(x, y):
    return D0 * (1.0 - (x**2 + y**2) / L**2)


def bowl_case(n, precision=synth.FP64):
    """The square [-1.5 L, 1.5 L]^2 (land walls) holding the bowl, the body at its t = 0 place."""
    mesh = synth.grid_mesh(n, n, 3.0 * L, 3.0 * L, seed=5, jitter=0.2)
    mesh.xy[:] -= 1.5 * L
    x, y = mesh.xy[:, 0], mesh.xy[:, 1]
    hb = bowl(x, y)
    init = np.zeros((3, mesh.n_nodes))
    init[0] = np.maximum(exact_zeta(x, 0.0), H0 - hb)  # dry land rests at depth h0
    return mesh, hb, synth.default_params(limiter=1, h0=H0, precision=precision), init


def wet_interior_error(mesh, u, t):
    """Mean and max |zeta_00 - zeta_exact| over elements whose exact depth exceeds 0.5 m."""
    c = mesh.xy[mesh.tri].mean(axis=1)  # the plane's element mean is its barycentre value
    ze = exact_zeta(c[:, 0], t)
    wet = ze + bowl(c[:, 0], c[:, 1]) > 0.5
    err = np.abs(u[0, 0] - ze)[wet]
    return err.mean(), err.max(), np.abs(ze[wet]).max()


def half_period_error(n, flux=0, p=1):
    mesh, hb, prm, init = bowl_case(n)
    prm["flux"] = flux
    prm["p"] = p
    o = oracle.Oracle(mesh, hb, prm, init_nodal=init, omp=True)  # bitwise the serial build
    steps = int(round(np.pi / W / o.dt))
    o.step(steps)
    return wet_interior_error(mesh, o.state(), steps * o.dt)


@pytest.mark.parametrize("flux,p", [(0, 1), (1, 1), (0, 2)])  # LLF / Roe at p = 1, LLF at p = 2
def test_thacker_planar_oscillation_converges(flux, p):
    m24, x24, amp = half_period_error(24, flux, p)
    m48, x48, _ = half_period_error(48, flux, p)
    assert amp > 1.5                      # the plane spans metres: a body left in place is far off
    assert m48 < 0.08 and x48 < 0.35      # LLF 0.051, 0.25 m (0.018, 0.091 at n = 96); Roe 0.043, 0.23;
                                          # p = 2 0.051, 0.23 (the front bounds the order)
    assert m24 / m48 > 2.0 and x24 / x48 > 2.0   # convergence faster than first order in h


# ------------------------------------------------------------------ with rotation
# With the Coriolis terms (+f q_y in x, -f q_x in y) the same bowl holds a body whose centre
# circles at r_c(t) = eta exp(i s t) (complex x + i y) while the fluid moves uniformly with its
# centre, u + i v = i s r_c.  The momentum equations u_t - f v + g zeta_x = 0 and
# v_t + f u + g zeta_y = 0 with zeta = (2 D0 / L^2) Re(r conj(r_c)) - D0 eta^2 / L^2 require
# s^2 + f s - w^2 = 0, i.e. s = (-f + sqrt(f^2 + 4 w^2)) / 2; continuity holds as without rotation.
OMEGA_EARTH = 7.2921e-5  # rad/s


def rotating_case(n, lat_deg=90.0, precision=synth.FP64):
    """Mesh, bathymetry, parameters, initial nodal state and the exact surface zeta(x, y, t, rate)
    of the rotating body; rate s (and the non-rotating w for comparison)."""
    f = 2.0 * OMEGA_EARTH * np.sin(np.radians(lat_deg))
    s = 0.5 * (-f + np.sqrt(f * f + 4.0 * W * W))

    def zeta(x, y, t, rate):
        rc = ETA * np.exp(1j * rate * t)
        return (2.0 * D0 / L**2) * (x * rc.real + y * rc.imag) - D0 * ETA**2 / L**2

    mesh = synth.grid_mesh(n, n, 3.0 * L, 3.0 * L, seed=5, jitter=0.2)
    mesh.xy[:] -= 1.5 * L
    x, y = mesh.xy[:, 0], mesh.xy[:, 1]
    hb = bowl(x, y)
    z0 = zeta(x, y, 0.0, s)
    wet = z0 + hb > 0.0
    init = np.zeros((3, mesh.n_nodes))
    init[0] = np.where(wet, z0, H0 - hb)
    init[2] = np.where(wet, (z0 + hb) * s * ETA, 0.0)  # q_y = H v(0), v(0) = s eta
    prm = synth.default_params(limiter=1, h0=H0, coriolis=1, coriolis_lat_deg=lat_deg, precision=precision)
    return mesh, hb, prm, init, zeta, s


def rotating_error(n):
    mesh, hb, prm, init, zeta, s = rotating_case(n)
    o = oracle.Oracle(mesh, hb, prm, init_nodal=init, omp=True)
    steps = int(round(np.pi / s / o.dt))  # half a turn
    o.step(steps)
    t = steps * o.dt
    c = mesh.xy[mesh.tri].mean(axis=1)
    ze = zeta(c[:, 0], c[:, 1], t, s)
    inner = ze + bowl(c[:, 0], c[:, 1]) > 0.5
    err = np.abs(o.state()[0, 0] - ze)[inner]
    without = np.abs(zeta(c[:, 0], c[:, 1], t, W) - ze)[inner]  # the same body if f were ignored
    return err.mean(), without.mean()


def test_thacker_rotating_body_converges():
    m24, _ = rotating_error(24)
    m48, rot = rotating_error(48)
    assert m48 < 0.08                   # measured 0.056 m (0.024 at n = 96)
    assert m24 / m48 > 2.0
    assert rot > 2.0 * m48              # the rotation's effect (0.139 m) is resolved


@pytest.mark.gpu
def test_thacker_gpu_fp64_matches_oracle_and_mixed_tracks_the_plane():
    from paper_2508_21208_gb300 import Model

    mesh, hb, prm, init = bowl_case(48)
    ref = oracle.Oracle(mesh, hb, prm, init_nodal=init)
    gpu = Model(mesh, hb, prm, init_nodal=init)
    assert abs(gpu.dt - ref.dt) <= 1e-14 * ref.dt
    steps = int(round(np.pi / W / ref.dt))
    ref.step(steps)
    gpu.step(steps)
    a, b = gpu.state(), ref.state()
    for v in range(3):
        assert np.linalg.norm(a[v] - b[v]) <= 1e-12 * np.linalg.norm(b[v]), v
    assert np.array_equal(gpu.flags(), ref.flags())
    _, _, prm32, _ = bowl_case(48, precision=synth.FP32_MIXED)
    mixed = Model(mesh, hb, prm32, init_nodal=init)
    mixed.step(steps)
    m64, x64, _ = wet_interior_error(mesh, b, steps * ref.dt)
    m32, x32, _ = wet_interior_error(mesh, mixed.state(), steps * ref.dt)
    print(f"STATED thacker n=48 steps={steps}: FP64 mean/max {m64:.4f}/{x64:.4f} m, "
          f"mixed {m32:.4f}/{x32:.4f} m")
    assert m32 < 1.05 * m64 + 1e-3 and x32 < 1.05 * x64 + 1e-3


@pytest.mark.gpu
def test_thacker_roe_gpu_fp64_matches_oracle():
    from paper_2508_21208_gb300 import Model

    mesh, hb, prm, init = bowl_case(32)
    prm["flux"] = 1
    ref = oracle.Oracle(mesh, hb, prm, init_nodal=init)
    gpu = Model(mesh, hb, prm, init_nodal=init)
    steps = int(round(np.pi / W / ref.dt))
    ref.step(steps)
    gpu.step(steps)
    a, b = gpu.state(), ref.state()
    for v in range(3):
        assert np.linalg.norm(a[v] - b[v]) <= 1e-12 * np.linalg.norm(b[v]), v
    assert np.array_equal(gpu.flags(), ref.flags())


@pytest.mark.gpu
def test_thacker_rotating_gpu_fp64_matches_oracle():
    from paper_2508_21208_gb300 import Model

    mesh, hb, prm, init, _, s = rotating_case(48)
    ref = oracle.Oracle(mesh, hb, prm, init_nodal=init)
    gpu = Model(mesh, hb, prm, init_nodal=init)
    steps = int(round(np.pi / s / ref.dt))
    ref.step(steps)
    gpu.step(steps)
    a, b = gpu.state(), ref.state()
    for v in range(3):
        assert np.linalg.norm(a[v] - b[v]) <= 1e-12 * np.linalg.norm(b[v]), v
    assert np.array_equal(gpu.flags(), ref.flags())
