"""Pins of the oracle's discretisation against closed forms, invariants and brute force.

Each test names what fixes the expected value: the PDE (Sec. 2.1, Eq. SWE), the weak form
(Sec. 2.2, Eq. elem_weak_form), or an exact solution of a special case.
"""
import math

import numpy as np
import pytest
from scipy import integrate
from scipy.special import eval_jacobi, eval_legendre

import oracle
from paper_2508_21208_gb300 import synth

G = 9.81


def _mesh_area(mesh):
    return 1.0


# ------------------------------------------------------------------ lake at rest
@pytest.mark.parametrize("p", [1, 2])
@pytest.mark.parametrize("zeta0", [0.0, 0.3])
def test_lake_at_rest_rhs_and_200_steps(zeta0, p):
    c = synth.config1(lake=True)
    c.params["p"] = p
    c.init_nodal[0] = zeta0
    o = oracle.Oracle(c.mesh, c.bathy, c.params, init_nodal=c.init_nodal)
    r = o.rhs(0.0)
    # the pressure gradient scale g H |grad h_b| ~ 9.81 * 12 * 2 pi / 1000 ~ 0.7 m/s^2
    assert np.abs(r).max() <= 1e-13 * 0.7 * 12.0
    o.step(200)
    u = o.state()
    assert np.abs(u[1:]).max() < 1e-11          # momentum stays at round-off
    assert np.abs(u[0, 0] - zeta0).max() < 1e-12


@pytest.mark.parametrize("p", [1, 2])
def test_mass_conserved_all_land_200_steps(p):
    c = synth.config1()
    c.params["p"] = p
    o = oracle.Oracle(c.mesh, c.bathy, c.params, init_nodal=c.init_nodal)
    m0, v0 = o.mass()
    o.step(200)
    m1, v1 = o.mass()
    assert abs(v1 - v0) <= 1e-14 * v0
    assert abs(m1 - m0) <= 1e-14 * v0


@pytest.mark.parametrize("p", [1, 2])
def test_mass_conserved_with_wetdry_and_limiter(p):
    c = synth.config2(n=24, p=p)
    c.mesh.bedge_type[:] = synth.BC_LAND  # closed basin
    c.params["tide_amp"] = 0.0
    # a slope-driven wave running up the shore
    x = c.mesh.xy[:, 0]
    c.init_nodal[0] = np.where(c.bathy > 0, 0.5 * np.exp(-((x - 80e3) / 5e3) ** 2), c.init_nodal[0])
    o = oracle.Oracle(c.mesh, c.bathy, c.params, init_nodal=c.init_nodal)
    m0, v0 = o.mass()
    o.step(200)
    m1, v1 = o.mass()
    assert abs(v1 - v0) <= 1e-14 * v0
    f = o.flags()
    assert (f == 2).sum() > 0 and (f == 0).sum() > 0


# ------------------------------------------------------------------ symmetry
def _mirrored_config1(n=20):
    rng = np.random.default_rng(5)
    left = rng.random((n, n // 2)) < 0.5
    flip = np.zeros((n, n), bool)
    flip[:, : n // 2] = left
    flip[:, n // 2:] = ~left[:, ::-1]   # mirroring about x = L/2 swaps the diagonal
    L = 1000.0
    mesh = synth.grid_mesh(n, n, L, L, 0, flip=flip)
    c = synth.config1(n=n)
    c.mesh = mesh
    x, y = mesh.xy[:, 0], mesh.xy[:, 1]
    c.bathy = 10.0 + 2.0 * np.sin(np.pi * x / L)
    c.init_nodal = np.zeros((3, mesh.n_nodes))
    c.init_nodal[0] = 0.1 * np.exp(-((x - 400.0) ** 2 + (y - 500.0) ** 2) / 100.0 ** 2) \
        + 0.1 * np.exp(-((x - 600.0) ** 2 + (y - 500.0) ** 2) / 100.0 ** 2)
    return c


@pytest.mark.parametrize("p", [1, 2])
def test_mirror_symmetry_about_x(p):
    c = _mirrored_config1()
    c.params["p"] = p
    o = oracle.Oracle(c.mesh, c.bathy, c.params, init_nodal=c.init_nodal)
    o.step(50)
    u = o.state()
    cen = c.mesh.xy[c.mesh.tri].mean(axis=1)
    key = {(round(a, 6), round(b, 6)): e for e, (a, b) in enumerate(cen)}
    mirror = np.array([key[(round(1000.0 - a, 6), round(b, 6))] for a, b in cen])
    scale = np.abs(u[:, 0]).max(axis=1)
    assert np.abs(u[0, 0] - u[0, 0, mirror]).max() <= 1e-13 * scale[0]
    assert np.abs(u[1, 0] + u[1, 0, mirror]).max() <= 1e-13 * scale[1]
    assert np.abs(u[2, 0] - u[2, 0, mirror]).max() <= 1e-13 * scale[2]
    assert scale[1] > 1e-3  # the flow is not trivial


# ------------------------------------------------------------------ source ODEs
def _uniform_case(params, q0, n=4):
    # 10 km cells keep the large explicit dt of these tests well inside the stability limit
    mesh = synth.grid_mesh(n, n, 40e3, 40e3, 9)
    hb = np.full(mesh.n_nodes, 10.0)
    init = np.zeros((3, mesh.n_nodes))
    init[1], init[2] = q0
    prm = synth.default_params(**params)
    return mesh, hb, init, prm


def _run_with_exact_ghost(mesh, hb, init, prm, hand_rk2, nsteps):
    """Boundary ghosts equal the uniform state of the current stage (known from the hand RK2),
    so the spatial operator vanishes and only the source terms act."""
    o = oracle.Oracle(mesh, hb, prm, init_nodal=init)
    dt = o.dt
    q = np.array([init[1, 0], init[2, 0]])
    for n in range(nsteps):
        q1, qn = hand_rk2(q, dt, n)

        def bnd(t, xy, a=q, b=q1, tn=n * dt):
            w = a if abs(t - tn) < 1e-9 * max(1.0, tn) else b
            out = np.zeros((len(xy), 3))
            out[:, 1], out[:, 2] = w
            return out

        o.set_mms(lambda t, xy: np.zeros((len(xy), 3)), bnd)
        o.step(1)
        q = qn
    return o


def test_quadratic_friction_matches_scalar_rk2():
    cf, H = 0.0025, 10.0
    mesh, hb, init, prm = _uniform_case(dict(friction=synth.FRICTION_QUADRATIC, cf=cf, dt=5.0), (1.0, -0.5))

    def f(q):
        return -cf * np.hypot(*q) * q / H ** 2

    def rk2(q, dt, n):
        q1 = q + dt * f(q)
        return q1, 0.5 * q + 0.5 * (q1 + dt * f(q1))

    o = _run_with_exact_ghost(mesh, hb, init, prm, rk2, 40)
    q = np.array([1.0, -0.5])
    for n in range(40):
        q = rk2(q, 5.0, n)[1]
    u = o.state()
    assert np.allclose(u[1, 0], q[0], rtol=1e-13, atol=0)
    assert np.allclose(u[2, 0], q[1], rtol=1e-13, atol=0)
    assert np.abs(u[1:, 1:]).max() < 1e-14
    assert abs(q[0] - 1.0) > 1e-3  # friction did act


def test_manning_friction_matches_scalar_rk2():
    """Manning's law tau_b = g n^2 |q| / H^(7/3) on a uniform flow (Sec. 2.1, Eq. SWE friction term)
    against the same SSP-RK2 written out by hand."""
    n, H, g = 0.02, 10.0, 9.81
    mesh, hb, init, prm = _uniform_case(dict(friction=synth.FRICTION_MANNING, manning_n=n, dt=5.0), (1.0, -0.5))

    def f(q):
        return -g * n * n * np.hypot(*q) * q / H ** (7.0 / 3.0)

    def rk2(q, dt, k):
        q1 = q + dt * f(q)
        return q1, 0.5 * q + 0.5 * (q1 + dt * f(q1))

    o = _run_with_exact_ghost(mesh, hb, init, prm, rk2, 40)
    q = np.array([1.0, -0.5])
    for k in range(40):
        q = rk2(q, 5.0, k)[1]
    u = o.state()
    assert np.allclose(u[1, 0], q[0], rtol=1e-13, atol=0)
    assert np.allclose(u[2, 0], q[1], rtol=1e-13, atol=0)
    assert abs(q[0] - 1.0) > 1e-3  # friction did act
    # Manning and quadratic friction agree when C_f = g n^2 / H^(1/3)
    prm_q = dict(prm, friction=synth.FRICTION_QUADRATIC, cf=g * n * n / H ** (1.0 / 3.0))
    oq = _run_with_exact_ghost(mesh, hb, init, prm_q, rk2, 40)
    assert np.allclose(oq.state()[1:, 0], u[1:, 0], rtol=1e-12, atol=0)


def test_coriolis_rotation_matches_rk2_amplification():
    lat = 28.0
    f = 2 * 7.2921e-5 * math.sin(math.radians(lat))
    dt = 50.0
    mesh, hb, init, prm = _uniform_case(dict(coriolis=1, coriolis_lat_deg=lat, dt=dt), (0.7, 0.2))
    A = np.array([[1 - (f * dt) ** 2 / 2, f * dt], [-f * dt, 1 - (f * dt) ** 2 / 2]])

    def rk2(q, dt_, n):
        q1 = q + dt_ * f * np.array([q[1], -q[0]])
        return q1, A @ q

    o = _run_with_exact_ghost(mesh, hb, init, prm, rk2, 30)
    q = np.linalg.matrix_power(A, 30) @ np.array([0.7, 0.2])
    u = o.state()
    assert np.allclose(u[1, 0], q[0], rtol=1e-13, atol=1e-15)
    assert np.allclose(u[2, 0], q[1], rtol=1e-13, atol=1e-15)


def test_uniform_wind_gives_constant_acceleration():
    vt, hd = 8.0, math.radians(30.0)
    prm = dict(hurricane=1, pc_hpa=1013.0, pn_hpa=1013.0, vt_ms=vt, track_heading=hd,
               track_x0=20e3, track_y0=20e3, coriolis_lat_deg=0.0, dt=20.0)
    mesh, hb, init, p = _uniform_case(prm, (0.0, 0.0))
    U = 0.5 * vt * np.array([math.cos(hd), math.sin(hd)])
    Um = np.hypot(*U)
    tau = 1.15 / 1000.0 * (0.75 + 0.067 * Um) * 1e-3 * Um * U   # Garratt drag, rho_a/rho_w

    def rk2(q, dt, n):
        return q + dt * tau, q + dt * tau

    o = _run_with_exact_ghost(mesh, hb, init, p, rk2, 10)
    u = o.state()
    assert np.allclose(u[1, 0], 10 * 20.0 * tau[0], rtol=1e-12)
    assert np.allclose(u[2, 0], 10 * 20.0 * tau[1], rtol=1e-12)


def test_holland_profile_at_rmax():
    mesh = synth.grid_mesh(10, 10, 100e3, 100e3, 0)
    hb = np.full(mesh.n_nodes, 100.0)
    prm = synth.default_params(hurricane=1, pc_hpa=950.0, pn_hpa=1013.0, rmax_m=40e3, holland_b=1.5,
                               vt_ms=0.0, track_x0=0.0, track_y0=0.0, coriolis_lat_deg=28.0)
    o = oracle.Oracle(mesh, hb, prm)
    F = o.forcing(0.0)
    node = int(np.argmin(np.hypot(mesh.xy[:, 0] - 40e3, mesh.xy[:, 1])))
    dp = (1013.0 - 950.0) * 100.0
    assert F[2, node] == pytest.approx(dp * (math.exp(-1.0) - 1.0) / 1000.0, rel=1e-14)  # (p - pn) / rho_w
    f = 2 * 7.2921e-5 * math.sin(math.radians(28.0))
    V = math.sqrt(1.5 / 1.15 * dp * math.exp(-1.0) + (40e3 * f / 2) ** 2) - 40e3 * f / 2
    Us = 0.9 * V
    cd = min(0.75 + 0.067 * Us, 3.5) * 1e-3
    assert F[0, node] == pytest.approx(0.0, abs=1e-15)
    assert F[1, node] == pytest.approx(1.15 / 1000.0 * cd * Us * Us, rel=1e-13)  # counter-clockwise
    # far field: pressure tends to the ambient value (anomaly towards 0)
    far = int(np.argmax(np.hypot(mesh.xy[:, 0], mesh.xy[:, 1])))
    assert F[2, node] < F[2, far] < 0.0


# ------------------------------------------------------------------ brute force
MODES = [(0, 0), (1, 0), (0, 1)]


def _psi(i, j, xi, eta):
    a = 2.0 * (1.0 + xi) / (1.0 - eta) - 1.0 if eta < 1.0 else -1.0
    return eval_legendre(i, a) * ((1.0 - eta) / 2.0) ** i * eval_jacobi(j, 2 * i + 1, 0, eta)


def _two_elements():
    xy = np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 1.0], [0.0, 1.0]]) * 50.0
    tri = np.array([[0, 1, 2], [0, 2, 3]], np.int32)
    bedge = np.array([[0, 1], [1, 2], [2, 3], [3, 0]], np.int32)
    return synth.Mesh(xy=xy, tri=tri, bedge=bedge, bedge_type=np.zeros(4, np.int32))


def _brute_rhs(mesh, hb_nodes, modes, prm):
    """Independent assembly of M^-1 [ (grad phi, F) + (phi, s) - <phi, LLF.n> ] with adaptive quadrature."""
    g = prm["g"]
    fcor = 2 * 7.2921e-5 * math.sin(math.radians(prm["coriolis_lat_deg"])) if prm["coriolis"] else 0.0
    X = mesh.xy
    out = np.zeros((3, 3, 2))
    elems = []
    for e, t in enumerate(mesh.tri):
        P0, P1, P2 = X[t[0]], X[t[1]], X[t[2]]
        J = np.column_stack([(P1 - P0) / 2, (P2 - P0) / 2])
        Ji = np.linalg.inv(J)
        hbv = hb_nodes[t]

        def ref(p, P0=P0, Ji=Ji):
            r = Ji @ (np.asarray(p) - P0)
            return r[0] - 1.0, r[1] - 1.0

        # bathymetry as the plane through the three vertex values
        A = np.column_stack([X[t], np.ones(3)])
        cb = np.linalg.solve(A, hbv)
        elems.append(dict(t=t, J=J, Ji=Ji, ref=ref, cb=cb, detJ=np.linalg.det(J)))

    def state(e, p):
        xi, eta = elems[e]["ref"](p)
        phi = np.array([_psi(i, j, xi, eta) for i, j in MODES])
        return modes[:, :, e] @ phi

    def hb(e, p):
        cb = elems[e]["cb"]
        return cb[0] * p[0] + cb[1] * p[1] + cb[2]

    def gradphi(e, k):
        # d psi/d(xi,eta) of the linear modes, mapped by J^-T
        d = [np.array([0.0, 0.0]), np.array([1.0, 0.5]), np.array([0.0, 1.5])][k]
        return elems[e]["Ji"].T @ d

    def flux(w, h):
        z, qx, qy = w
        H = z + h
        P = 0.5 * g * (H * H - h * h)
        return np.array([[qx, qy], [qx * qx / H + P, qx * qy / H], [qx * qy / H, qy * qy / H + P]])

    def src(w, e, p):
        z, qx, qy = w
        H = z + hb(e, p)
        cb = elems[e]["cb"]
        tau = prm["cf"] * math.hypot(qx, qy) / H ** 2
        return np.array([0.0, g * z * cb[0] - tau * qx + fcor * qy, g * z * cb[1] - tau * qy - fcor * qx])

    def llf(wi, wo, h, n):
        Fi, Fo = flux(wi, h) @ n, flux(wo, h) @ n
        Hi, Ho = wi[0] + h, wo[0] + h
        lam = max(abs(wi[1:] @ n) / Hi + math.sqrt(g * Hi), abs(wo[1:] @ n) / Ho + math.sqrt(g * Ho))
        return 0.5 * (Fi + Fo) - 0.5 * lam * (wo - wi)

    for e, E in enumerate(elems):
        t = E["t"]
        P0, P1, P2 = X[t[0]], X[t[1]], X[t[2]]
        for v in range(3):
            for k in range(3):
                def integrand(s, r):
                    p = P0 + r * (P1 - P0) + s * (P2 - P0)
                    w = state(e, p)
                    F = flux(w, hb(e, p))
                    xi, eta = E["ref"](p)
                    phik = _psi(*MODES[k], xi, eta)
                    return (gradphi(e, k) @ F[v] + phik * src(w, e, p)[v]) * 4 * E["detJ"]
                val, _ = integrate.dblquad(integrand, 0, 1, 0, lambda r: 1 - r, epsabs=1e-13, epsrel=1e-13)
                out[v, k, e] += val
        # edges of e, outward normal; the neighbour (if any) shares the edge
        for a in range(3):
            na, nb = t[a], t[(a + 1) % 3]
            Pa, Pb = X[na], X[nb]
            tv = Pb - Pa
            L = np.linalg.norm(tv)
            n = np.array([tv[1], -tv[0]]) / L
            other = [f for f in range(len(elems)) if f != e and na in elems[f]["t"] and nb in elems[f]["t"]]
            for v in range(3):
                for k in range(3):
                    def integ(s):
                        p = Pa + s * tv
                        wi = state(e, p)
                        h = hb(e, p)
                        if other:
                            wo = state(other[0], p)
                        else:
                            qn = wi[1:] @ n
                            wo = np.array([wi[0], *(wi[1:] - 2 * qn * n)])
                        xi, eta = E["ref"](p)
                        return llf(wi, wo, h, n)[v] * _psi(*MODES[k], xi, eta) * L
                    val, _ = integrate.quad(integ, 0, 1, epsabs=1e-12, epsrel=1e-12, limit=200)
                    out[v, k, e] -= val
        norms = np.array([2.0, 1.0 / 3.0, 1.0])
        out[:, :, e] /= E["detJ"] * norms[None, :]
    return out


def test_two_element_rhs_polynomial_case_exact():
    """q = 0 and zeta continuous: every integrand is a polynomial, so quadrature is exact."""
    mesh = _two_elements()
    hbn = np.array([10.0, 10.5, 11.0, 10.2])
    zn = np.array([0.1, -0.2, 0.05, 0.3])  # nodal zeta -> continuous linear pieces
    init = np.zeros((3, 4))
    init[0] = zn
    prm = synth.default_params(friction=synth.FRICTION_QUADRATIC, cf=0.0025, dt=1.0)
    o = oracle.Oracle(mesh, hbn, prm, init_nodal=init)
    got = o.rhs(0.0)
    ref = _brute_rhs(mesh, hbn, o.state(), prm)
    assert np.allclose(got, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_two_element_rhs_general_case():
    """Discontinuous random state with momentum: LLF dissipation, advection, friction, Coriolis."""
    mesh = _two_elements()
    hbn = np.array([10.0, 10.5, 11.0, 10.2])
    rng = np.random.default_rng(3)
    modal = np.zeros((3, 3, 2))
    modal[0] = 0.2 * rng.standard_normal((3, 2))
    modal[1:] = 0.5 * rng.standard_normal((2, 3, 2))
    prm = synth.default_params(friction=synth.FRICTION_QUADRATIC, cf=0.0025, coriolis=1,
                               coriolis_lat_deg=30.0, dt=1.0)
    o = oracle.Oracle(mesh, hbn, prm, init_modal=modal)
    got = o.rhs(0.0)
    ref = _brute_rhs(mesh, hbn, modal, prm)
    # the oracle's fixed rules integrate rational / kinked integrands only approximately
    assert np.allclose(got, ref, rtol=0, atol=1e-4 * np.abs(ref).max())
    # a sign or index slip anywhere would be O(1): check the deviation is far below that
    assert np.abs(got - ref).max() < 1e-3 * np.abs(ref).max()


# ------------------------------------------------------------------ tide
def test_tidal_signal_arrives_at_shallow_water_speed():
    n = 80
    mesh = synth.grid_mesh(n, 4, 20e3, 1e3, 4, open_sides=("left",))
    hb = np.full(mesh.n_nodes, 10.0)
    prm = synth.default_params(tide_amp=0.01, tide_period=44714.0, dt=2.0)
    o = oracle.Oracle(mesh, hb, prm)
    T = 1000.0
    o.step(int(T / 2.0))
    u = o.state()
    cx = mesh.xy[mesh.tri].mean(axis=1)[:, 0]
    z0 = 0.01 * math.sin(2 * math.pi * T / 44714.0)
    reached = cx[u[0, 0] > 0.01 * z0]
    front = reached.max()
    c = math.sqrt(G * 10.0)
    h = 20e3 / n
    assert abs(front - c * T) < 2 * h


def test_dt_single_triangle_closed_form():
    xy = np.array([[0.0, 0.0], [3.0, 0.0], [0.0, 4.0]])
    mesh = synth.Mesh(xy=xy, tri=np.array([[0, 1, 2]], np.int32), bedge=np.zeros((0, 2), np.int32),
                      bedge_type=np.zeros(0, np.int32))
    hb = np.full(3, 2.0)
    for p, fac in ((1, 1.0), (2, 3.0 / 5.0)):
        prm = synth.default_params(p=p, cfl=0.3)
        o = oracle.Oracle(mesh, hb, prm)
        r = 1.0  # inradius of the 3-4-5 triangle
        assert o.dt == pytest.approx(0.3 * fac * r / math.sqrt(G * 2.0), rel=1e-15)


def test_invalid_mesh_rejected():
    mesh = _two_elements()
    bad = synth.Mesh(xy=mesh.xy, tri=mesh.tri[:, ::-1].copy(), bedge=mesh.bedge, bedge_type=mesh.bedge_type)
    with pytest.raises(ValueError):
        oracle.Oracle(bad, np.full(4, 10.0), synth.default_params())


def test_edge_counts_of_grid_mesh():
    for n in (3, 7):
        c = synth.config1(n=n)
        o = oracle.Oracle(c.mesh, c.bathy, c.params, init_nodal=c.init_nodal)
        assert o.n_edges == 3 * n * n + 2 * n
        assert o.n_edges - o.n_interior == 4 * n


def _gradient_balance_residual(ncell, lat=28.0, rho_a=1.15, rho_w=1000.0):
    """Largest |V^2/r + f V - (1/rho_a) dp/dr| / max|(1/rho_a) dp/dr| along a line of nodes 5-300 km
    from a stationary vortex: V from the oracle's surface stress inverted through the Garratt drag
    law (|U| = 0.9 V), dp/dr by central differences of its pressure anomaly (node spacing
    295.5 km / ncell).  Also returns the largest V."""
    from scipy.optimize import brentq

    mesh = synth.grid_mesh(ncell, 1, 300e3 - 4.5e3, 50.0, 0)
    mesh.xy[:, 0] += 5e3
    prm = synth.default_params(hurricane=1, pc_hpa=950.0, pn_hpa=1013.0, rmax_m=40e3, holland_b=1.5,
                               vt_ms=0.0, track_x0=0.0, track_y0=0.0, coriolis_lat_deg=lat,
                               rho_air=rho_a, rho_water=rho_w)
    F = oracle.Oracle(mesh, np.full(mesh.n_nodes, 100.0), prm).forcing(0.0)
    line = np.where(mesh.xy[:, 1] == 0.0)[0]
    line = line[np.argsort(mesh.xy[line, 0])]
    r = mesh.xy[line, 0]
    tx, ty, pa = F[0, line], F[1, line], F[2, line]
    assert np.all(np.abs(tx) <= 1e-12 * np.abs(ty)) and np.all(ty > 0)  # tangential, counter-clockwise
    f = 2 * 7.2921e-5 * math.sin(math.radians(lat))

    def surface_wind(kk):  # C_d(|U|) |U|^2 = kk
        return brentq(lambda u: min(0.75 + 0.067 * u, 3.5) * 1e-3 * u * u - kk, 0.0, 200.0, xtol=1e-14)

    V = np.array([surface_wind(kk) for kk in ty * rho_w / rho_a]) / 0.9
    rhs = rho_w * (pa[2:] - pa[:-2]) / (r[2:] - r[:-2]) / rho_a  # p - pn = rho_w * anomaly
    lhs = V[1:-1] ** 2 / r[1:-1] + f * V[1:-1]
    return np.abs(lhs - rhs).max() / np.abs(rhs).max(), V.max()


def test_holland_wind_and_pressure_in_gradient_balance():
    """The vortex's wind and pressure fields satisfy the gradient-wind balance at every radius:
    Holland's gradient wind is the positive root of V^2 / r + f V = (1/rho_a) dp/dr.  The residual
    is the central differences' truncation error: it shrinks fourfold when the spacing halves."""
    coarse, _ = _gradient_balance_residual(985)
    fine, vmax = _gradient_balance_residual(1970)
    assert fine < 1e-4                    # measured 6.7e-5 (2.7e-4 at twice the spacing)
    assert coarse / fine > 3.5            # second-order differencing error, not a model mismatch
    assert vmax > 40.0                    # a hurricane-strength vortex


def test_openmp_build_is_bitwise_the_serial_build():
    """The oracle's OpenMP build (used for the large cases and the CPU baseline) parallelises
    only loops whose iterations write disjoint data, so it reproduces the serial build exactly."""
    c = synth.config2(n=24)
    c.params["hurricane"] = 1
    c.params["coriolis"] = 1
    c.params["coriolis_lat_deg"] = 28.0
    runs = []
    for omp in (False, True):
        o = oracle.Oracle(c.mesh, c.bathy, c.params, init_nodal=c.init_nodal, omp=omp)
        o.step(60)
        runs.append((o.state(), o.flags(), o.mass()))
    assert np.array_equal(runs[0][0], runs[1][0])
    assert np.array_equal(runs[0][1], runs[1][1])
    assert runs[0][2] == runs[1][2]
