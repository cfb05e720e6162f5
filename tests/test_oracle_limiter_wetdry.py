"""Invariants that pin the oracle's slope limiter and wet/dry operator (Sec. 5.2.3 SLOPELIM,
WETDRY).  The paper does not define either operator, so beyond these properties their parity is
unpinned: the limiter is the Cockburn-Shu triangle minmod limiter, the wet/dry step a
mean-preserving vertex-depth fix.  Vertex values are evaluated here with scipy's Jacobi
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
