"""The similarity law of Sec. II on the CUDA path, at the full size of the throughput workload.

Scaling the pressure by 2, the lengths and the time step by 1/2, the density by 4 and the field by
2 changes every input by an exact power of two, so the particle step follows the same trajectory
in cell units bit for bit (the oracle is pinned to this in test_oracle_similarity.py).  This is a
property that holds at any size: it checks the 2e7-particle neon column in the launch
configuration of the benchmark (MIXED storage, persistent step kernel, periodic sort) without an
oracle run at that size."""
import numpy as np
import pytest

import paper_2202_03215_gb300 as pb
from paper_2202_03215_gb300 import build as pbuild
from paper_2202_03215_gb300 import workloads as w
from tests.test_oracle_similarity import SAME, scaled

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    pbuild.build()


def _same(g1: dict, g2: dict, where: str) -> None:
    for k in ("n_e", "n_i", "step", "next_id"):
        assert g1[k] == g2[k], (where, k)
    for k in SAME:
        a, b = g1[k], g2[k]
        if not np.array_equal(a, b):
            bad = np.nonzero(a != b)[0]
            raise AssertionError(f"{where} {k}: {len(bad)} differ, first {bad[:5]}")
    assert np.array_equal(g2["E"], 2.0 * g1["E"]), f"{where}: E"


def test_full_size_neon_column_and_its_similar_column():
    # the homogeneous state of eq. 2 for R = 1 cm carrying 1 mA, rounded (any field and density
    # give the same test)
    p1 = w.config_neon_column(drive=w.DRIVE_E0, E0_Vpm=645.6, n0_m3=2.2e14, sort_every=250)
    p2 = scaled(p1, 2.0)
    c1, c2 = pb.Column(p1), pb.Column(p2)
    _same(c1.get_state(), c2.get_state(), "init")
    c1.step(12)   # two ion pushes
    c2.step(12)
    _same(c1.get_state(), c2.get_state(), "step 12")
    c1.step(248)  # through the sort at step 250
    c2.step(248)
    _same(c1.get_state(), c2.get_state(), "step 260")
    s1, s2 = c1.stats(), c2.stats()
    assert s1["n_coll_e"] == s2["n_coll_e"] and s1["n_coll_i"] == s2["n_coll_i"]
    assert sum(s1["n_coll_e"]) > 10**6
