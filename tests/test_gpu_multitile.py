"""Parity of the particle step's full launch pipeline with the oracle over many steps.

At 2e6 electrons and 2e6 ions each of the 152 persistent CTAs walks about 13
tiles of 1024 particles, so the asynchronous two-tile staging, the candidate
queues carried across tiles, the shared-memory bins over a cell window and the
global fall-back for particles outside the window (the first steps start from
the unsorted initial state) all run, together with sorts of both species, ion
pushes and paired removals (Sec. II).  Every fifth step the whole state is
compared bit for bit: cells, offsets, velocities, ids, node charges, field,
counts and the collision and birth counters.
"""
import numpy as np
import pytest

import oracle
import paper_2202_03215_gb300 as pb
from paper_2202_03215_gb300 import build as pbuild
from paper_2202_03215_gb300 import workloads as w
from tests.test_gpu_parity import assert_same

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    pbuild.build()


@pytest.mark.parametrize("precision", [w.MIXED, w.FP64])
def test_multi_tile_multi_step_neon_column_bit_exact(precision):
    n = 2_000_000 if precision == w.MIXED else 600_000
    p = w.config_neon_column(n_per_species=n, precision=precision, sort_every=5, seed=5)
    g = pb.Column(p)
    o = oracle.Oracle(p)
    s0 = o.get_state()
    assert_same(g.get_state(), s0, "init")
    # start at step 41: steps 41..44 run on the unsorted initial state (global deposit
    # fall-back), electrons are sorted at 45, 50, ..., ions at 50, ions pushed at 50, 60, 70
    s0["step"] = 41
    g.set_state(s0)
    o.set_state(s0)
    c0g, c0o = g.stats(), o.stats()
    for k in range(6):
        g.step(5)
        o.step(5)
        assert_same(g.get_state(), o.get_state(), f"step {41 + 5 * (k + 1)}")
    sg, so = g.stats(), o.stats()

    def delta(a, b, key):
        return np.asarray(a[key], dtype=np.int64) - np.asarray(b[key], dtype=np.int64)

    for key in ("births", "n_coll_e", "n_coll_i", "overflow_e", "overflow_i"):
        assert np.array_equal(delta(sg, c0g, key), delta(so, c0o, key)), key
    assert delta(sg, c0g, "births") > 0 and delta(sg, c0g, "n_coll_i").sum() > 0
    g.close()
