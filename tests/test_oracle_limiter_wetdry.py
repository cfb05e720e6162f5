"""Invariants and hand-worked examples that pin the oracle's slope limiter and wet/dry operator
(Sec. 5.2.3 SLOPELIM, WETDRY).  The paper does not define either operator: the limiter is the
Cockburn-Shu triangle minmod limiter, the wet/dry step a mean-preserving vertex-depth fix.  Vertex values are evaluated here with scipy's Jacobi
polynomials, independently of the oracle's basis code."""
import numpy as np
import pytest
from scipy.special import eval_jacobi, eval_legendre

import oracle
from paper_2508_21208_gb300 import synth


def _psi_lin(xi, eta):
    a = 2.0 * (1.0 + xi) / (1.0 - eta) - 1.0 if eta < 1.0 else -1.0
    return np.array([1.0, eval_legendre(1, a) * (1.0 - eta) / 2.0, eval_jacobi(1, 1, 0, eta)])


VERT = np.array([_psi_lin(-1.0, -1.0), _psi_lin(1.0, -1.0), _psi_lin(-1.0, 1.0)])   # [vertex, mode]
MID = np.array([_psi_lin(0.0, 0.0), _psi_lin(-1.0, 0.0), _psi_lin(0.0, -1.0)])       # edge midpoints


def _random_state(c, rng, amp=0.3):
    o = oracle.Oracle(c.mesh, c.bathy, c.params, init_nodal=c.init_nodal)
    u = o.state()
    u[:, :3] += amp * rng.standard_normal(u[:, :3].shape) * np.array([1.0, 0.3, 0.3])[None, :, None]
    return o, u


def _small_shelf(n=20):
    c = synth.config2(n=n)
    return c


# ------------------------------------------------------------------ limiter
def test_limiter_keeps_means_and_shrinks_midpoint_deviations():
    c = _small_shelf()
    c.params["h0"] = 0.0  # limiter alone
    rng = np.random.default_rng(1)
    o, u = _random_state(c, rng)
    u[0, 0] += 60.0  # keep depth positive everywhere
    o.set_state(u)
    o.apply_limiter()
    w = o.state()
    assert np.array_equal(w[:, 0], u[:, 0])                      # element means untouched
    before = np.einsum("mk,vke->vme", MID[:, 1:], u[:, 1:3])      # linear-part deviations
    after = np.einsum("mk,vke->vme", MID[:, 1:], w[:, 1:3])
    assert np.all(np.abs(after) <= np.abs(before) + 1e-12)
    assert np.all((after == 0) | (np.sign(after) == np.sign(before)) | (np.abs(after) < 1e-12))
    assert np.abs(after - before).max() > 1e-3                    # it did limit something


def test_limiter_leaves_linear_field_unchanged_away_from_boundary():
    c = _small_shelf()
    c.params["h0"] = 0.0
    x, y = c.mesh.xy[:, 0], c.mesh.xy[:, 1]
    nodal = np.zeros((3, c.mesh.n_nodes))
    nodal[0] = 1e-5 * x - 2e-5 * y + 3.0
    nodal[1] = 2e-6 * x + 1.0
    nodal[2] = -1e-6 * y
    o = oracle.Oracle(c.mesh, c.bathy, c.params, init_nodal=nodal)
    u = o.state()
    o.apply_limiter()
    w = o.state()
    # elements whose three neighbours exist (interior) see exact linear reconstructions
    tri = c.mesh.tri
    xy = c.mesh.xy
    on_bnd = (np.isclose(xy[:, 0], 0) | np.isclose(xy[:, 0], 100e3) | np.isclose(xy[:, 1], 0)
              | np.isclose(xy[:, 1], 50e3))
    interior = ~on_bnd[tri].any(axis=1)
    scale = np.abs(u[:, 1:3]).max()
    assert np.abs(w[:, :, interior] - u[:, :, interior]).max() <= 1e-9 * scale


def test_limiter_p2_drops_quadratic_modes_only_where_active():
    c = synth.config2(n=12, p=2)
    c.params["h0"] = 0.0
    rng = np.random.default_rng(2)
    o = oracle.Oracle(c.mesh, c.bathy, c.params, init_nodal=c.init_nodal)
    u = o.state()
    u[0, 0] += 60.0
    sub = rng.random(u.shape[2]) < 0.5      # only half the elements get slopes
    u[:, 1:3, sub] += 0.2 * rng.standard_normal(u[:, 1:3, sub].shape)
    u[:, 3:] += 0.05 * rng.standard_normal(u[:, 3:].shape)
    o.set_state(u)
    o.apply_limiter()
    w = o.state()
    changed = np.any(w[:, 1:3] != u[:, 1:3], axis=(0, 1))
    assert changed.any() and (~changed).any()
    assert np.all(w[:, 3:, changed] == 0.0)
    assert np.array_equal(w[:, 3:, ~changed], u[:, 3:, ~changed])


# ------------------------------------------------------------------ wet/dry
def _vertex_depth(u, c):
    zv = np.einsum("ik,ke->ie", VERT, u[0, :3])        # [vertex, elem]
    return zv + c.bathy[c.mesh.tri].T


def test_wetdry_invariants():
    c = _small_shelf()
    rng = np.random.default_rng(4)
    o, u = _random_state(c, rng, amp=0.5)
    o.set_state(u)
    o.apply_wetdry()
    w = o.state()
    f = o.flags()
    h0 = c.params["h0"]
    assert np.array_equal(w[0, 0], u[0, 0])          # mean surface kept
    Hv = _vertex_depth(w, c)
    Hm = Hv.mean(axis=0)
    assert set(np.unique(f)) == {0, 1, 2}
    dry, wet = f == 2, f == 0
    assert np.all(Hv[:, ~dry] >= h0 - 1e-12)         # positivity where water is kept
    assert np.all(Hv[:, wet] > h0 + 1e-10)
    assert np.abs(Hv[:, dry] - Hm[dry]).max() < 1e-12  # dry elements are flat
    assert np.all(w[1:, :, dry] == 0.0)              # and carry no momentum
    # already-wet linear elements are untouched
    Hu = _vertex_depth(u, c)
    untouched = np.all(Hu > h0, axis=0)
    assert np.array_equal(w[:, :, untouched], u[:, :, untouched])
    # idempotent
    o.apply_wetdry()
    w2 = o.state()
    assert np.allclose(w2, w, rtol=0, atol=1e-12)
    assert np.array_equal(o.flags(), f)


def test_initial_shelf_state_dry_land_at_h0():
    c = _small_shelf(n=64)  # cells narrow enough that whole elements lie on land (x > 96 km)
    o = oracle.Oracle(c.mesh, c.bathy, c.params, init_nodal=c.init_nodal)
    f = o.flags()
    cx = c.mesh.xy[c.mesh.tri].mean(axis=1)[:, 0]
    land = np.all(c.bathy[c.mesh.tri] < 0, axis=1)
    sea = np.all(c.bathy[c.mesh.tri] > 0.5, axis=1)
    assert np.all(f[land] == 2)
    assert np.all(f[sea] == 0)
    assert cx[f == 2].min() > 90e3


# ---------------------------------------------------------------- hand-worked examples
def _modes_from_vertices(a0, a1, a2):
    """Linear Dubiner modes of the interpolant through vertex values (a0, a1, a2): the mean, then
    psi_10 and psi_01 coefficients (psi_10 = -1, 1, 0 and psi_01 = -1, -1, 2 at the vertices)."""
    return np.array([(a0 + a1 + a2) / 3.0, 0.5 * (a1 - a0), (2.0 * a2 - a0 - a1) / 6.0])


def _vertices_from_modes(m):
    return np.array([m[0] - m[1] - m[2], m[0] + m[1] - m[2], m[0] + 2.0 * m[2]])


def test_limiter_worked_example():
    """Cockburn-Shu limiting of one element, worked by hand.

    Four triangles split the triangle (0,0), (2,0), (0,2) at its edge midpoints D(1,0), E(1,1),
    F(0,1); the centre element DEF has neighbours DBE, FEC, ADF across DE, EF, FD.  Each midpoint
    of the centre, measured from its barycentre (2/3, 2/3), is half the vector to the barycentre
    of the neighbour across that edge, so the neighbour-mean difference at each midpoint is half
    the difference of the means.

    Centre: mean 1, vertex values D 1.2, E 1.4, F 0.4, i.e. midpoint deviations 0.3 (DE), -0.1 (EF),
    -0.2 (FD).  Neighbour means: DBE 1.2, FEC 0.7, ADF 0.9, i.e. differences 0.1, -0.15, -0.05.
    minmod(deviation, 1.5 x difference): 0.15, -0.1, -0.075; their sum -0.025 != 0, so the
    negative ones are scaled by 0.15 / 0.175 = 6/7: 0.15, -0.6/7, -0.45/7.  The limited vertex
    values follow: D = 1 + 1.2/7, E = 1 + 0.9/7, F = 0.7.
    """
    xy = np.array([[0, 0], [2, 0], [0, 2], [1, 0], [1, 1], [0, 1]], float) * 1000.0
    tri = np.array([[3, 4, 5], [0, 3, 5], [3, 1, 4], [5, 4, 2]], np.int32)
    bedge = np.array([[0, 3], [3, 1], [1, 4], [4, 2], [2, 5], [5, 0]], np.int32)
    mesh = synth.Mesh(xy, tri, bedge, np.zeros(6, np.int32))
    hb = np.full(6, 10.0)
    prm = synth.default_params(limiter=1)
    u = np.zeros((3, 3, 4))
    u[0, :, 0] = _modes_from_vertices(1.2, 1.4, 0.4)
    u[0, 0, 1], u[0, 0, 2], u[0, 0, 3] = 0.9, 1.2, 0.7  # ADF, DBE, FEC: means only
    o = oracle.Oracle(mesh, hb, prm, init_modal=u)
    o.set_state(u)
    o.apply_limiter()
    got = _vertices_from_modes(o.state()[0, :, 0])
    assert np.allclose(got, [1.0 + 1.2 / 7.0, 1.0 + 0.9 / 7.0, 0.7], rtol=0, atol=1e-14)
    assert o.state()[0, 0, 0] == pytest.approx(1.0, abs=1e-15)  # mean kept
    # the same element with every deviation inside the neighbour bounds is left alone
    u2 = u.copy()
    u2[0, :, 0] = _modes_from_vertices(1.04, 1.06, 0.9)  # deviations 0.05, -0.02, -0.03
    o.set_state(u2)
    o.apply_limiter()
    assert np.allclose(o.state()[0, :, 0], u2[0, :, 0], rtol=0, atol=1e-15)


def test_wetdry_worked_example():
    """The wetting/drying operator on one element, worked by hand (h0 = 0.01 m).

    Vertex depths (0.005, 0.02, 0.05): mean 0.025 > h0, vertex 0 lifted to h0, the others' excess
    over h0 (0.01, 0.04) scaled by 3 (0.025 - 0.01) / 0.05 = 0.9 to keep the mean:
    (0.01, 0.019, 0.046).  The element is partially wet; with beds (-0.5, 0.3, 1.0) the mean
    surface (-0.2417 m) lies below the highest bed among the vertices at h0 (0.5 m, vertex 0), so
    its momentum is removed.  Vertex depths (0.002, 0.004, 0.006): mean 0.004 <= h0, dry: flat at
    0.004 with no momentum.
    """
    xy = np.array([[0.0, 0.0], [1000.0, 0.0], [0.0, 1000.0]])
    mesh = synth.Mesh(xy, np.array([[0, 1, 2]], np.int32), np.array([[0, 1], [1, 2], [2, 0]], np.int32),
                      np.zeros(3, np.int32))
    hb = np.array([-0.5, 0.3, 1.0])
    prm = synth.default_params(h0=0.01)
    for H, expect, flag in (((0.005, 0.02, 0.05), (0.01, 0.019, 0.046), 1),
                            ((0.002, 0.004, 0.006), (0.004, 0.004, 0.004), 2)):
        u = np.zeros((3, 3, 1))
        u[0, :, 0] = _modes_from_vertices(*(np.array(H) - hb))
        u[1, :, 0] = [0.3, 0.01, -0.02]
        u[2, :, 0] = [-0.1, 0.0, 0.03]
        o = oracle.Oracle(mesh, hb, prm, init_modal=u)
        o.set_state(u)
        o.apply_wetdry()
        s = o.state()
        got = _vertices_from_modes(s[0, :, 0]) + hb
        assert np.allclose(got, expect, rtol=0, atol=1e-15), (H, got)
        assert o.flags()[0] == flag
        assert np.all(s[1:] == 0.0)


def test_wetdry_edge_rule_worked_example():
    """The edge rule between a wet and a dry element (reading of Sec. 5.2.2): the edge carries no
    flow unless the wet side's surface at the edge's Gauss points rises above the edge's highest
    bed.  Two triangles share the diagonal (1000, 0)-(0, 1000) of a square; the dry one (upper
    right) is land up to 1 m above the datum (h_b = -1 there, -0.6 on the shared edge), water at
    h0.  The wet one (lower left) is level at its mean surface zeta_A: below the highest bed on
    the edge (0.6 m), no mass reaches the dry element; above it, mass flows in."""
    xy = np.array([[0.0, 0.0], [1000.0, 0.0], [0.0, 1000.0], [1000.0, 1000.0]])
    tri = np.array([[0, 1, 2], [1, 3, 2]], np.int32)
    bedge = np.array([[0, 1], [1, 3], [3, 2], [2, 0]], np.int32)
    mesh = synth.Mesh(xy, tri, bedge, np.zeros(4, np.int32))
    hb = np.array([5.0, -0.6, -0.6, -1.0])
    prm = synth.default_params(h0=0.01)
    for zeta_a, flows in ((0.4, False), (0.9, True)):
        u = np.zeros((3, 3, 2))
        u[0, 0, 0] = zeta_a                                   # wet, level
        u[0, :, 1] = _modes_from_vertices(*(0.01 - hb[[1, 3, 2]]))  # dry, water at h0
        o = oracle.Oracle(mesh, hb, prm, init_modal=u)
        o.set_state(u)
        assert list(o.flags()) == [1, 2] or list(o.flags()) == [0, 2]
        L = o.rhs(0.0)
        if flows:
            assert L[0, 0, 1] > 1e-6 and L[0, 0, 0] < -1e-9   # mass leaves A, enters B
        else:
            assert L[0, 0, 1] == 0.0 and abs(L[0, 0, 0]) < 1e-15


PAIR_ORDER = ((0, 1), (2, 0), (1, 2))  # (i, i+1), (i+2, i), (i+1, i+2) as offsets from i


def _limit_from_geometry(xy, tri, u, nu=1.5, order=PAIR_ORDER):
    """The Cockburn-Shu limiter of every element (p = 1), recomputed from the coordinates alone.

    Independent of the oracle's preprocessing: neighbours come from shared vertex pairs, the
    barycentre directions and boundary mirror images from vector geometry, each edge midpoint's
    decomposition from numpy.linalg.solve (pairs tried in the stated order (i,i+1), (i+2,i),
    (i+1,i+2); none gives no slope bound), midpoint values from scipy's basis table MID, and the
    rebuilt linear modes from a 2x2 solve through the midpoints of edges 0 and 1.  Also returns
    the largest number of admissible pairs found for one midpoint.
    """
    ne = tri.shape[0]
    nbr = -np.ones((ne, 3), dtype=int)
    seen = {}
    for e in range(ne):
        for l in range(3):
            key = tuple(sorted((int(tri[e, (l + 1) % 3]), int(tri[e, (l + 2) % 3]))))
            if key in seen:
                f, lf = seen.pop(key)
                nbr[e, l], nbr[f, lf] = f, e
            else:
                seen[key] = (e, l)
    bary = xy[tri].mean(axis=1)
    rebuild = np.linalg.inv(MID[:2, 1:])  # midpoint deviations of edges 0, 1 -> (psi_10, psi_01)
    out = u.copy()
    most = 0
    for e in range(ne):
        P, b0 = xy[tri[e]], bary[e]
        mids, dirs = [], []
        for l in range(3):
            A, B = P[(l + 1) % 3], P[(l + 2) % 3]
            mids.append(0.5 * (A + B) - b0)
            if nbr[e, l] >= 0:
                dirs.append(bary[nbr[e, l]] - b0)
            else:
                t = (B - A) / np.linalg.norm(B - A)
                foot = A + t * np.dot(b0 - A, t)
                dirs.append(2.0 * (foot - b0))
        weights = []
        for i in range(3):
            admissible = []
            for o1, o2 in order:
                j1, j2 = (i + o1) % 3, (i + o2) % 3
                M = np.column_stack([dirs[j1], dirs[j2]])
                if abs(np.linalg.det(M)) < 1e-12 * np.linalg.norm(M) ** 2:
                    continue
                a = np.linalg.solve(M, mids[i])
                if a.min() >= -1e-10:
                    admissible.append((j1, j2, a))
            most = max(most, len(admissible))
            weights.append(admissible[0] if admissible else None)
        for v in range(3):
            ub = u[v, 0, e]
            means = [u[v, 0, nbr[e, l]] if nbr[e, l] >= 0 else ub for l in range(3)]
            dev = MID[:, 1:] @ u[v, 1:3, e]
            d = np.empty(3)
            for i in range(3):
                bound = 0.0
                if weights[i] is not None:
                    j1, j2, a = weights[i]
                    bound = a[0] * (means[j1] - ub) + a[1] * (means[j2] - ub)
                x, y = dev[i], nu * bound
                d[i] = min(x, y) if (x > 0 and y > 0) else (max(x, y) if (x < 0 and y < 0) else 0.0)
            if np.all(d == dev):
                continue
            pos, neg = d[d > 0].sum(), -d[d < 0].sum()
            tp = min(1.0, neg / pos) if pos > 0 else 0.0
            tm = min(1.0, pos / neg) if neg > 0 else 0.0
            dh = np.where(d > 0, tp * d, np.where(d < 0, tm * d, 0.0))
            out[v, 1:3, e] = rebuild @ dh[:2]
    return out, most


@pytest.mark.parametrize("seed", [3, 4])
def test_limiter_equals_geometric_recomputation_on_skewed_mesh(seed):
    """On a jittered mesh (non-aligned neighbours, skewed cones, boundary mirrors on every side)
    the oracle's limiter equals the recomputation from coordinates, element by element.  Every
    midpoint there has exactly one admissible neighbour pair, so the order of trial never decides;
    the boundary mirror rule does (a shifted mirror image, or a zero mean behind a boundary edge,
    fails this test)."""
    mesh = synth.grid_mesh(12, 9, 12e3, 9e3, seed=seed, jitter=0.3)
    hb = np.full(mesh.n_nodes, 20.0)
    prm = synth.default_params(limiter=1)
    rng = np.random.default_rng(seed)
    ne = mesh.n_elems
    u = np.zeros((3, 3, ne))
    u[:, 0] = rng.standard_normal((3, ne)) * np.array([0.5, 2.0, 2.0])[:, None]
    u[:, 1:3] = rng.standard_normal((3, 2, ne)) * np.array([0.4, 1.5, 1.5])[:, None, None]
    o = oracle.Oracle(mesh, hb, prm, init_modal=u)
    o.set_state(u)
    o.apply_limiter()
    got = o.state()
    want, most = _limit_from_geometry(mesh.xy, mesh.tri, u)
    assert most == 1
    changed = np.any(want[:, 1:3] != u[:, 1:3], axis=1)
    assert changed.sum() > ne // 2                      # most variables were limited
    assert np.array_equal(got[:, 0], u[:, 0])           # means kept
    scale = np.abs(u[:, 1:3]).max()
    assert np.abs(got - want).max() <= 1e-12 * scale


def test_limiter_pair_order_worked_example():
    """The order in which neighbour pairs are tried decides, worked by hand.

    Centre element A(0,0) B(12,0) C(5,1) (km), barycentre b0 = (17/3, 1/3); neighbours across
    BC, CA and AB have third vertices (16,4), (13,8) and (9,-3), so the barycentre directions are
    d0 = (16/3, 4/3), d1 = (1/3, 8/3), d2 = (4/3, -4/3).  The midpoint of edge 0 (BC), at
    m0 - b0 = (17/6, 1/6), decomposes with non-negative weights along two pairs:
    (d2, d0) with (13/40, 9/20) and (d1, d2) with (1, 15/8); the pair (d0, d1) fails (-13/62).
    Tried in the order (i,i+1), (i+2,i), (i+1,i+2), edge 0 takes (d2, d0).  Edge 1 has no
    admissible pair (its bound is 0); edge 2 has two that both put 1/4 on d2 alone.

    Surface: centre mean 0 and linear modes (0.2, 0.6), i.e. midpoint deviations 0.4, 0.2, -0.6;
    neighbour means 1.0, 0.0, -0.8.  Bounds (nu = 1.5): edge 0, 1.5 (13/40 (-0.8) + 9/20 (1.0)) =
    0.285; edge 1, 0; edge 2, 1.5 (1/4)(-0.8) = -0.3.  minmod: 0.285, 0, -0.3; their sum is
    negative, so the negative part is scaled by 0.285/0.3: deviations 0.285, 0, -0.285, i.e.
    linear modes (0.285, 0.285).  With (d1, d2) at edge 0 the bound there would be
    1.5 (1 (0.0) + 15/8 (-0.8)) = -2.25, minmod 0, and the element would be flattened.
    """
    km = 1000.0
    xy = np.array([[0, 0], [12, 0], [5, 1], [16, 4], [13, 8], [9, -3]], float) * km
    tri = np.array([[0, 1, 2], [2, 1, 3], [0, 2, 4], [1, 0, 5]], np.int32)
    bedge = np.array([[1, 3], [3, 2], [2, 4], [4, 0], [0, 5], [5, 1]], np.int32)
    mesh = synth.Mesh(xy, tri, bedge, np.zeros(6, np.int32))
    hb = np.full(6, 20.0)
    prm = synth.default_params(limiter=1)
    u = np.zeros((3, 3, 4))
    u[0, :, 0] = [0.0, 0.2, 0.6]
    u[0, 0, 1:] = [1.0, 0.0, -0.8]
    assert np.allclose(MID[:, 1:] @ u[0, 1:3, 0], [0.4, 0.2, -0.6], atol=1e-15)
    o = oracle.Oracle(mesh, hb, prm, init_modal=u)
    o.set_state(u)
    o.apply_limiter()
    got = o.state()
    assert np.allclose(got[0, :, 0], [0.0, 0.285, 0.285], rtol=0, atol=1e-14)
    # the recomputation from coordinates agrees in the stated order and differs in any order that
    # tries (i+1, i+2) before (i+2, i)
    want, most = _limit_from_geometry(mesh.xy, mesh.tri, u)
    assert most == 2
    assert np.allclose(want[0, :, 0], got[0, :, 0], rtol=0, atol=1e-14)
    for order in (((0, 1), (1, 2), (2, 0)), ((1, 2), (2, 0), (0, 1))):
        alt, _ = _limit_from_geometry(mesh.xy, mesh.tri, u, order=order)
        assert np.allclose(alt[0, 1:3, 0], [0.0, 0.0], atol=1e-14)


def test_wetdry_edge_rule_keeps_a_dry_bank_dry_while_water_sloshes():
    """The edge rule in motion: water moving in a wet element against a dry bank element.

    The shared edge runs from A (bed at the datum) to B (bed 1 m above it); the wet element W
    below it deepens to 5.5 m at its third vertex, and the dry bank D above it rises to 2 m, with
    its water at h0.  W's surface starts tilted up towards B (0.5 m at A, 1.05 m at B: wet
    everywhere) and then sloshes back.  At the edge's Gauss points W's surface stays below the
    edge's highest bed (1 m), so the edge is closed: D must stay exactly as it is and W must keep
    its water, while W's water moves.  Letting every edge flow (removing the rule, planted in a
    scratch copy of the oracle) moves water into D in the first step, since W's surface at the
    edge lies well above D's (h0 above the bed)."""
    xy = np.array([[0.0, 0.0], [1000.0, 0.0], [500.0, -1000.0], [500.0, 1000.0]])
    tri = np.array([[0, 2, 1], [0, 1, 3]], np.int32)  # W = (A, E, B), D = (A, B, C)
    bedge = np.array([[0, 2], [2, 1], [1, 3], [3, 0]], np.int32)
    mesh = synth.Mesh(xy, tri, bedge, np.zeros(4, np.int32))
    hb = np.array([0.0, -1.0, 5.0, -2.0])       # h_b positive down: bed elevations 0, 1, -5, 2 m
    prm = synth.default_params(h0=0.01)
    u = np.zeros((3, 3, 2))
    u[0, :, 0] = _modes_from_vertices(0.5, 0.5, 1.05)           # W at its vertices A, E, B
    u[0, :, 1] = _modes_from_vertices(*(0.01 - hb[[0, 1, 3]]))  # D at h0 depth
    o = oracle.Oracle(mesh, hb, prm, init_modal=u)
    o.set_state(u)
    assert list(o.flags()) == [0, 2]
    area = 0.5 * 1000.0 * 1000.0
    d0 = o.state()[:, :, 1].copy()
    w_mass = o.state()[0, 0, 0] * area
    s, _ = oracle.edge_rule(2)
    bed_top = 1.0
    moved, w_flags = 0.0, set()
    for _ in range(40):
        z = o.state()[0, :, 0]
        zA, zB = z[0] - z[1] - z[2], z[0] + 2.0 * z[2]  # W's surface at A and B (vertices 0 and 2)
        traces = zA + (zB - zA) * 0.5 * (1.0 + s)
        assert traces.max() < bed_top                  # the edge stays closed
        o.step(1)
        st = o.state()
        assert np.array_equal(st[:, :, 1], d0)          # the bank is untouched
        f = o.flags()
        assert f[1] == 2 and f[0] in (0, 1)            # W may dry at B as it sloshes back
        w_flags.add(int(f[0]))
        assert abs(st[0, 0, 0] * area - w_mass) <= 1e-12 * w_mass
        moved = max(moved, np.abs(st[1:, 0, 0]).max())
    assert moved > 1e-3                                 # W's water does move
