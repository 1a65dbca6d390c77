"""Many collision processes per species (up to 16): a synthetic neon with its excitation
spread over seven levels (the shape of a multi-level cross-section set) stepped on the
GPU against the oracle, bit for bit, with every level's collision count compared."""
import numpy as np
import pytest

import oracle
import paper_2202_03215_gb300 as pb
from paper_2202_03215_gb300 import build as pbuild
from paper_2202_03215_gb300 import workloads as w

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    pbuild.build()


@pytest.mark.parametrize("precision", [w.FP64, w.MIXED])
def test_seven_level_neon_matches_the_oracle(precision):
    p = w.config_neon_column(n_per_species=20_000, precision=precision, E0_Vpm=3000.0, n_cells=1024,
                             sort_every=0).with_(xsec=w.neon_multilevel_xsecs(), Te0_eV=8.0)
    g, o = pb.Column(p), oracle.Oracle(p)
    for k in range(3):
        g.step(10)
        o.step(10)
        a, b = g.get_state(), o.get_state()
        for key in a:
            if isinstance(a[key], np.ndarray):
                assert np.array_equal(a[key], b[key]), (k, key)
    sg, so = g.stats(), o.stats()
    assert sg["n_coll_e"] == so["n_coll_e"]
    assert sum(1 for c in sg["n_coll_e"][1:8] if c > 0) >= 5      # most of the seven levels were hit
    assert sg["births"] == so["births"]
    g.close()
