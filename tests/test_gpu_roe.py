"""Roe numerical flux on the GPU (Sec. 2.2: the paper allows LLF or Roe) against the oracle."""
import numpy as np
import pytest

import oracle
from paper_2508_21208_gb300 import Model, synth
from paper_2508_21208_gb300.dgswem import VARIANT_FUSED, VARIANT_SPLIT, VARIANT_TILED

pytestmark = pytest.mark.gpu


def rel(a, b):
    return max(np.linalg.norm(a[v] - b[v]) / max(np.linalg.norm(b[v]), 1e-300) for v in range(3))


CASES = {
    "shelf": lambda: synth.config2(n=40),
    "storm": lambda: synth.config3(n=32),
    "shelf_p2": lambda: synth.config2(n=20, p=2),
}


@pytest.mark.parametrize("variant", [VARIANT_SPLIT, VARIANT_FUSED, VARIANT_TILED])
@pytest.mark.parametrize("name", list(CASES))
def test_roe_parity(name, variant):
    c = CASES[name]()
    c.params["flux"] = synth.FLUX_ROE
    g = Model(c.mesh, c.bathy, c.params, init_nodal=c.init_nodal, variant=variant, block=128)
    o = oracle.Oracle(c.mesh, c.bathy, c.params, init_nodal=c.init_nodal, omp=True)
    assert g.dt == pytest.approx(o.dt, rel=1e-14)
    g.step(80)
    o.step(80)
    assert rel(g.state(), o.state()) <= 1e-12
    assert np.array_equal(g.flags(), o.flags())
