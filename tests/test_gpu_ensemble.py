"""Batched ensemble: every member must equal the same scenario run alone (bitwise, same tiled kernels),
FP64 members must match the oracle, and the bounded grid barrier must turn a withheld arrival into
DGSWEM_ETIMEOUT instead of a hang."""
import time

import numpy as np
import pytest

import oracle
from paper_2508_21208_gb300 import Ensemble, Model, synth
from paper_2508_21208_gb300.dgswem import ENSEMBLE_PERSISTENT, ENSEMBLE_PHASED, VARIANT_TILED, DgswemError

pytestmark = pytest.mark.gpu


def small_ensemble(precision):
    """Three storms on two basin meshes of different size (member 0 and 2 share a mesh)."""
    meshes, bathys, members = synth.ensemble(members_per_mesh=1, mesh_n=(20, 28), precision=precision)
    extra = synth.storm_track(1002)
    prm = dict(members[0][1])
    prm.update(extra)
    members.append((0, prm, None))
    for _, p, _ in members:
        p["track_x0"] = 150e3  # keep the vortex over these small domains
        p["rmax_m"] = 60e3
    return meshes, bathys, members


@pytest.mark.parametrize("mode", [ENSEMBLE_PERSISTENT, ENSEMBLE_PHASED])
def test_members_equal_single_runs(mode):
    meshes, bathys, members = small_ensemble(synth.FP32_MIXED)
    ens = Ensemble(meshes, bathys, members, block=64, mode=mode)
    ens.step(25)
    for i, (mi, prm, _) in enumerate(members):
        # the ensemble's element phase is the tiled update with the tile size = block
        single = Model(meshes[mi], bathys[mi], prm, variant=VARIANT_TILED, block=64)
        assert ens.info(i)[0] == single.dt
        single.step(25)
        a, b = ens.state(i), single.state()
        assert np.array_equal(a, b), (i, np.abs(a - b).max())
        assert np.abs(a[1]).max() > 0.0


def test_fp64_members_match_oracle():
    meshes, bathys, members = small_ensemble(synth.FP64)
    ens = Ensemble(meshes, bathys, members, block=128, mode=ENSEMBLE_PERSISTENT)
    ens.step(30)
    for i, (mi, prm, _) in enumerate(members):
        o = oracle.Oracle(meshes[mi], bathys[mi], prm)
        assert ens.info(i)[0] == pytest.approx(o.dt, rel=1e-14)
        o.step(30)
        a, b = ens.state(i), o.state()
        for v in range(3):
            rel = np.linalg.norm(a[v] - b[v]) / max(np.linalg.norm(b[v]), 1e-300)
            assert rel <= 1e-12, (i, v, rel)


def test_autotuned_ensemble_runs():
    meshes, bathys, members = small_ensemble(synth.FP32_MIXED)
    ens = Ensemble(meshes, bathys, members)
    ens.step(5)
    ens.sync()
    kps, mode, block = ens.graph_info()
    assert mode in (ENSEMBLE_PERSISTENT, ENSEMBLE_PHASED) and block in (64, 128, 256)


def test_withheld_barrier_arrival_times_out():
    meshes, bathys, members = small_ensemble(synth.FP32_MIXED)
    ens = Ensemble(meshes, bathys, members, block=64, mode=ENSEMBLE_PERSISTENT)
    ens.step(2)
    ens.sync()
    ens.set_fault(True)
    t0 = time.time()
    ens.step(3)
    with pytest.raises(DgswemError) as ei:
        ens.sync()
    assert ei.value.code == -6  # DGSWEM_ETIMEOUT
    assert time.time() - t0 < 30.0
    # the device is still usable: a fresh ensemble runs
    ok = Ensemble(meshes, bathys, members, block=64, mode=ENSEMBLE_PERSISTENT)
    ok.step(2)
    ok.sync()


def test_fp64_one_storm_per_standard_mesh_matches_oracle():
    """One FP64 storm on each of the four ensemble meshes (49,928 / 199,712 / 399,618 / 798,848
    elements), batched in one launch, against the oracle after 20 steps."""
    meshes, bathys, members = synth.ensemble(members_per_mesh=1, precision=synth.FP64)
    ens = Ensemble(meshes, bathys, members, mode=ENSEMBLE_PERSISTENT)
    ens.step(20)
    for i, (mi, prm, _) in enumerate(members):
        o = oracle.Oracle(meshes[mi], bathys[mi], prm, omp=True)
        assert ens.info(i)[0] == pytest.approx(o.dt, rel=1e-14)
        o.step(20)
        a, b = ens.state(i), o.state()
        assert np.abs(b[1]).max() > 0.0  # the storm moved water
        for v in range(3):
            rel = np.linalg.norm(a[v] - b[v]) / max(np.linalg.norm(b[v]), 1e-300)
            assert rel <= 1e-12, (i, v, rel)


@pytest.mark.parametrize("p", [1, 2])
@pytest.mark.parametrize("mode", [ENSEMBLE_PERSISTENT, ENSEMBLE_PHASED])
def test_members_with_wetdry_fronts_equal_single_runs(mode, p):
    """Shelf scenarios with dry land and a tide (FP32-mixed): the ensemble updates and limits its
    wetting/drying front elements in double in its own front phases, and every member must equal
    the same scenario run alone (whose front goes through the model's front kernels) bit for bit,
    flags included."""
    cases = [synth.config2(n=24, p=p, precision=synth.FP32_MIXED),
             synth.config2(n=28, seed=5, p=p, precision=synth.FP32_MIXED)]
    meshes = [c.mesh for c in cases]
    bathys = [c.bathy for c in cases]
    members = [(0, cases[0].params, cases[0].init_nodal), (1, cases[1].params, cases[1].init_nodal),
               (0, dict(cases[0].params, tide_amp=0.3, tide_phase=1.0), cases[0].init_nodal)]
    ens = Ensemble(meshes, bathys, members, block=64, mode=mode)
    ens.step(40)
    for i, (mi, prm, init) in enumerate(members):
        single = Model(meshes[mi], bathys[mi], prm, init_nodal=init, variant=VARIANT_TILED, block=64)
        single.step(40)
        f = single.flags()
        assert (f == 1).any() and (f == 0).any() and (f == 2).any()  # a front exists
        assert np.array_equal(ens.flags(i), f), i
        a, b = ens.state(i), single.state()
        assert np.array_equal(a, b), (i, np.abs(a - b).max())
