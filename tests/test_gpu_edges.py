"""Edge cases of the particle step against the oracle, bit for bit, through the C ABI: empty
columns, particle counts around the number of CTAs and the 1024-particle tile, a column emptied by
radial losses, the smallest grid (3 cells) and particles that cross the periodic column several
times in one step (the modulo branch of the wrap, Sec. II periodic re-injection)."""
import numpy as np
import pytest

import oracle
import paper_2202_03215_gb300 as pb
from paper_2202_03215_gb300 import build as pbuild
from paper_2202_03215_gb300 import workloads as w
from tests.helpers import beam_state
from tests.test_gpu_parity import assert_same, small

pytestmark = pytest.mark.gpu

FORMS = [w.FP64, w.MIXED]


@pytest.fixture(scope="module", autouse=True)
def _built():
    pbuild.build()


def _run_both(p, chunks=(1, 11)):
    g, o = pb.Column(p), oracle.Oracle(p)
    assert_same(g.get_state(), o.get_state(), "init")
    for n in chunks:
        g.step(n)
        o.step(n)
        assert_same(g.get_state(), o.get_state(), f"step {o.get_state()['step']}")
    return g, o


@pytest.mark.parametrize("precision", FORMS)
def test_empty_column(precision):
    g, o = _run_both(small(precision, n_e0=0, n_i0=0), chunks=(1, 24))
    s = g.get_state()
    assert s["n_e"] == 0 and s["n_i"] == 0
    assert not s["Q_e"].any() and not s["Q_i"].any()


@pytest.mark.parametrize("precision", FORMS)
@pytest.mark.parametrize("n", [1, 151, 152, 153, 1023, 1025, 4097])
def test_counts_around_the_launch_shape(precision, n):
    # fewer particles than CTAs, one per CTA, a partial tile, one more than a tile
    _run_both(small(precision, n_e0=n, n_i0=n, capacity=2 * n + 64))


@pytest.mark.parametrize("precision", FORMS)
def test_radial_losses_empty_the_column(precision):
    # P_w = 1 - exp(-nu_w dt) = 0.5 per electron step (ions: dt_i = 10 dt, nearly all lost)
    p = small(precision, n_e0=3000, n_i0=3000, loss_mode=w.LOSS_RADIAL, nu_w=np.log(2.0) / 2e-11)
    g, o = _run_both(p, chunks=(1, 5, 30))
    s = g.get_state()
    assert s["n_e"] == 0 and s["n_i"] == 0
    g.step(3)
    o.step(3)
    assert_same(g.get_state(), o.get_state(), "empty, stepping on")


@pytest.mark.parametrize("precision", FORMS)
def test_three_cell_column(precision):
    _run_both(small(precision, n_e0=3000, n_i0=3000, n_cells=3), chunks=(1, 10, 9))


@pytest.mark.parametrize("precision", FORMS)
def test_particles_crossing_the_column_several_times(precision):
    """Electrons moving 3.7 column lengths per step and ions 2.5 per ion step, both directions:
    the wrap takes the remainder of a cell index far outside [0, N)."""
    n, N = 4000, 97
    p = w.Params(L_m=0.05, n_cells=N, dt_s=2e-11, field_mode=w.FIELD_APPLIED, drive=w.DRIVE_E0, E0_Vpm=0.0,
                 n_e0=n, n_i0=n, ion_subcycle=10, loss_mode=w.LOSS_NONE, precision=precision, seed=13,
                 capacity=4 * n)
    f32 = precision == w.MIXED
    rng = np.random.default_rng(17)
    st = beam_state(n, N, 3.7 * p.L_m / p.dt_s, rng, n_i=n, ion_speed=2.5 * p.L_m / (10 * p.dt_s), float32=f32)
    for sp in ("e", "i"):
        st[f"vx_{sp}"][::2] *= -1.0   # half of each species the other way
    g, o = pb.Column(p), oracle.Oracle(p)
    g.set_state(st)
    o.set_state(st)
    assert_same(g.get_state(), o.get_state(), "set")
    for k in (1, 10):   # an ion push at step 0 and step 10
        g.step(k)
        o.step(k)
        assert_same(g.get_state(), o.get_state(), f"step {k}")
    assert g.stats()["n_coll_e"] == o.stats()["n_coll_e"]
