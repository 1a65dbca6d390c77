"""Failures raised on the device and reported on the host, made by the inputs, not by a fault: more
births than particle slots gives PIC_ECAPACITY after the step (the births are not written), the
error latches on the handle, and the handle is still freed cleanly."""
import numpy as np
import pytest

import paper_2202_03215_gb300 as pb
from paper_2202_03215_gb300 import build as pbuild
from paper_2202_03215_gb300 import workloads as w
from tests.helpers import QE, ME, beam_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    pbuild.build()


@pytest.mark.parametrize("precision", [w.FP64, w.MIXED])
def test_births_beyond_capacity_raise_and_latch(precision):
    # a 60 eV electron beam in argon ionizes ~7 % per step: ~140 births against 10 free slots
    n = 2000
    p = w.Params(L_m=0.05, n_cells=100, dt_s=2e-11, field_mode=w.FIELD_APPLIED, drive=w.DRIVE_E0, E0_Vpm=0.0,
                 n_e0=n, n_i0=0, ion_subcycle=0, loss_mode=w.LOSS_NONE, precision=precision, capacity=n + 10)
    g = pb.Column(p)
    st = beam_state(n, p.n_cells, np.sqrt(2 * QE * 60.0 / ME), np.random.default_rng(2),
                    float32=precision == w.MIXED)
    g.set_state(st)
    with pytest.raises(pb.PicError) as ei:
        g.step(1)
    assert ei.value.code == -4 and "capacity" in str(ei.value)
    with pytest.raises(pb.PicError) as again:   # latched: the next call reports it too
        g.step(1)
    assert again.value.code == -4
    # a new state clears the error: 1800 particles leave 210 free slots for ~126 births
    m = 1800
    small = beam_state(m, p.n_cells, np.sqrt(2 * QE * 60.0 / ME), np.random.default_rng(3),
                       float32=precision == w.MIXED)
    g.set_state(small)
    g.step(1)
    s = g.stats()
    assert m < s["n_e"] <= p.capacity and s["n_i"] == s["n_e"] - m
    g.close()
