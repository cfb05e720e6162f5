"""The workloads at their full sizes and stated step counts, against the FP64 oracle.

- FP64 form: relative L2 <= 1e-12 on every state field and identical wet/dry flags after 2000
  steps of the 199,712-element shelf and 500 steps of the 3.2M-element storm domain.
- FP32-mixed form (float flux/source arithmetic, FP64 RK state, mass sums and wet/dry depth
  tests; the elements at the wetting/drying front in double): the largest surface-elevation
  difference at the element vertices must stay within 1e-4 m everywhere after 500 and 1000 steps
  of the shelf at p = 1 and p = 2, and after 1000 steps of one storm-ensemble member on each of the
  four ensemble meshes; the measured values (also the discharge differences, the wet/dry flag
  mismatches and the mass difference) are printed on lines starting with "STATED".
"""
import json

import numpy as np
import pytest

import oracle
from paper_2508_21208_gb300 import Ensemble, Model, synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

ZETA_BOUND_M = 1e-4


def rel_l2(a, b):
    return np.array([np.linalg.norm(a[v] - b[v]) / max(np.linalg.norm(b[v]), 1e-300) for v in range(3)])


def vertex_values(u, p):
    """Each field's value at the three vertices of every element, from its modes (3 x 3 x n)."""
    ph = np.array([oracle.basis(p, xi, eta)[0] for xi, eta in ((-1.0, -1.0), (1.0, -1.0), (-1.0, 1.0))])
    return np.einsum("ak,vke->vae", ph, u)


def tri_area(mesh):
    a = mesh.xy[mesh.tri[:, 1]] - mesh.xy[mesh.tri[:, 0]]
    b = mesh.xy[mesh.tri[:, 2]] - mesh.xy[mesh.tri[:, 0]]
    return 0.5 * np.abs(a[:, 0] * b[:, 1] - a[:, 1] * b[:, 0])


def report(tag, p, steps, a, b, mass_a, mass_b, vol, mesh, fa, fb):
    """Largest vertex differences over all elements and over the elements none of whose vertices
    touches a non-wet element in either run (away from the wetting/drying front)."""
    va, vb = vertex_values(a, p), vertex_values(b, p)
    ez = np.abs(va[0] - vb[0]).max(axis=0)
    eq = np.abs(va[1:] - vb[1:]).max(axis=(0, 1))
    front_node = np.zeros(mesh.n_nodes, bool)
    for f in (fa, fb):
        front_node[mesh.tri[f != 0].ravel()] = True
    interior = ~front_node[mesh.tri].any(axis=1)
    out = {"case": tag, "p": p, "steps": steps,
           "max_abs_zeta_err_m": float(ez.max()), "max_abs_q_err_m2s": float(eq.max()),
           "rms_zeta_err_m": float(np.sqrt(np.mean(ez ** 2))),
           "max_abs_zeta_err_away_from_wetdry_front_m": float(ez[interior].max()),
           "max_abs_q_err_away_from_wetdry_front_m2s": float(eq[interior].max()),
           "argmax_zeta_err_flags_gpu_oracle": [int(fa[ez.argmax()]), int(fb[ez.argmax()])],
           "argmax_zeta_err_x_m": float(mesh.xy[mesh.tri[ez.argmax()]].mean(axis=0)[0]),
           "flag_mismatches": int((fa != fb).sum()),
           "max_abs_q_m2s": float(np.abs(vb[1:]).max()),
           "mass_anomaly_diff_over_volume": (mass_a - mass_b) / vol}
    print("STATED " + json.dumps(out), flush=True)
    return out


def test_shelf_fp64_2000_steps():
    c = synth.config2()
    g = Model(c.mesh, c.bathy, c.params, init_nodal=c.init_nodal)
    o = oracle.Oracle(c.mesh, c.bathy, c.params, init_nodal=c.init_nodal, omp=True)
    g.step(2000)
    o.step(2000)
    err = rel_l2(g.state(), o.state())
    print("STATED " + json.dumps({"case": "shelf-199712 fp64", "steps": 2000, "rel_l2": err.tolist()}))
    assert np.all(err <= 1e-12), err
    assert np.array_equal(g.flags(), o.flags())


def test_storm_fp64_500_steps():
    c = synth.config3()
    g = Model(c.mesh, c.bathy, c.params, init_nodal=c.init_nodal)
    o = oracle.Oracle(c.mesh, c.bathy, c.params, init_nodal=c.init_nodal, omp=True)
    g.step(500)
    o.step(500)
    err = rel_l2(g.state(), o.state())
    print("STATED " + json.dumps({"case": "storm-3200450 fp64", "steps": 500, "rel_l2": err.tolist()}))
    assert np.all(err <= 1e-12), err
    assert np.array_equal(g.flags(), o.flags())


@pytest.mark.parametrize("p", [1, 2])
def test_shelf_mixed_error_500_1000(p):
    c = synth.config2(p=p, precision=synth.FP32_MIXED)
    g = Model(c.mesh, c.bathy, c.params, init_nodal=c.init_nodal)
    prm = dict(c.params)
    prm["precision"] = synth.FP64
    o = oracle.Oracle(c.mesh, c.bathy, prm, init_nodal=c.init_nodal, omp=True)
    out = []
    for steps in (500, 1000):
        g.step(500)
        o.step(500)
        mo, vol = o.mass()
        out.append(report("shelf-199712 mixed", p, steps, g.state(), o.state(), g.mass()[0], mo, vol,
                          c.mesh, g.flags(), o.flags()))
    for r in out:
        assert r["max_abs_zeta_err_m"] <= ZETA_BOUND_M
        assert r["flag_mismatches"] == 0
        assert abs(r["mass_anomaly_diff_over_volume"]) <= 1e-11


def test_ensemble_mixed_error_1000():
    """Eight storms (two per mesh of 49,928 / 199,712 / 399,618 / 798,848 elements) advanced
    together; the first storm on each mesh against the oracle, with the GPU's own wet/dry flags."""
    meshes, bathys, members = synth.ensemble(members_per_mesh=2)
    ens = Ensemble(meshes, bathys, members)
    ens.step(1000)
    for i in (0, 2, 4, 6):
        mi, prm, _ = members[i]
        prm = dict(prm)
        prm["precision"] = synth.FP64
        o = oracle.Oracle(meshes[mi], bathys[mi], prm, omp=True)
        o.step(1000)
        a, b = ens.state(i), o.state()
        mo, vol = o.mass()
        # the member's mass anomaly from its modes, on the host
        r = report(f"ensemble member {i} ({meshes[mi].n_elems} elements) mixed", 1, 1000, a, b,
                   float(np.sum(tri_area(meshes[mi]) * a[0, 0])), mo, vol, meshes[mi],
                   ens.flags(i), o.flags())
        assert r["max_abs_zeta_err_m"] <= ZETA_BOUND_M
        assert r["flag_mismatches"] == 0
