"""Batched columns (pic_init_batch / pic_step_batch): every column of a batch
evolves bit for bit like the same column advanced alone, through the
autotuning steps, the captured-graph cycles and the periodic sorts; and one
column against the CPU oracle directly."""
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


def _columns(precision, sort_every):
    cells = [97, 500, 2048, 3001]
    npart = [5000, 30000, 12000, 20000]
    out = []
    for c, (N, n) in enumerate(zip(cells, npart)):
        argon = c % 2 == 0
        out.append(w.Params(gas_mass_amu=w.AMU_AR if argon else w.AMU_NE, pressure_torr=0.5 + 0.5 * c,
                            L_m=0.02 * (c + 1), n_cells=N, dt_s=1e-11, ion_subcycle=10, drive=w.DRIVE_E0,
                            E0_Vpm=2000.0, V_applied=0.0, n_e0=n, n_i0=n, n0_m3=1e15 * (c + 1),
                            xsec=w.argon_xsecs(eps_max_e=200.0) if argon else w.neon_xsecs(),
                            eps_max_e_eV=200.0, precision=precision, sort_every=sort_every, seed=5,
                            capacity=2 * n, column=c))
    return out


@pytest.mark.parametrize("sort_every", [0, 7])
@pytest.mark.parametrize("precision", [w.FP64, w.MIXED])
def test_batched_columns_equal_lone_columns(precision, sort_every):
    params = _columns(precision, sort_every)
    b = pb.Batch(params)
    t = b.tune()   # the autotuner's steps (none when an equal batch was tuned before)
    tuned, me, mi = b.schedule()
    assert tuned and me in (1, 2, 3, 4, 6, 8) and mi in (1, 2, 3, 4, 6, 8)
    b.step(30)     # graph cycles where no sort falls
    lone = [pb.Column(p) for p in params]
    for c in lone:
        c.step(t + 30)
    for i, (bc, lc) in enumerate(zip(b.columns, lone)):
        assert_same(bc.get_state(), lc.get_state(), f"column {i}")
        assert bc.stats()["n_coll_e"] == lc.stats()["n_coll_e"]
    assert all(c.stats()["step"] == t + 30 for c in b.columns)
    assert sum(c.stats()["births"] for c in b.columns) > 0   # the births path ran inside the batch


def test_tuned_schedule_is_cached_by_batch_shape():
    # a batch of a shape tuned before in this process starts with that schedule (no tuning
    # steps); a batch of another shape tunes; the schedule never changes the columns' evolution
    params = _columns(w.MIXED, 0)
    a = pb.Batch(params)
    a.tune()
    tuned = a.schedule()
    a.close()
    b = pb.Batch(params)
    assert b.schedule() == tuned      # from the cache: tuned, the same multipliers
    b.step(5)
    c = pb.Batch(params[:3])          # another shape
    assert c.schedule()[0] is False
    c.close()
    lone = pb.Column(params[1])
    lone.step(5)
    assert_same(b.columns[1].get_state(), lone.get_state(), "cached schedule")
    b.close()


def test_batched_sort_matches_oracle():
    # the batched sort (one launch per radix phase for all columns) against the oracle's
    # counting sort: columns of 97 (one pass) to 3001 cells, several 4096-particle tiles each
    params = _columns(w.MIXED, 5)
    b = pb.Batch(params)
    b.step(16)
    for k in (0, 3):
        o = oracle.Oracle(params[k])
        o.step(16)
        assert_same(b.columns[k].get_state(), o.get_state(), f"column {k} vs oracle")


def test_batched_column_matches_oracle():
    params = _columns(w.MIXED, 0)
    b = pb.Batch(params)
    b.step(21)
    o = oracle.Oracle(params[2])
    o.step(21)
    assert_same(b.columns[2].get_state(), o.get_state(), "column 2 vs oracle")


def test_batched_sweep_workload_builds():
    cols = w.config_batch_sweep(n_columns=6, particle_scale=0.01)
    b = pb.Batch(cols)
    b.step(12)
    for c in b.columns:
        s = c.stats()
        assert s["step"] == 12 and s["n_e"] > 0
