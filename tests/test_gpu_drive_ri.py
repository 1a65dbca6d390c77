"""The (R, I) drive on the GPU: a column started with PIC_DRIVE_RI is the column
started with PIC_DRIVE_E0 at the field and density pic_drive_ri returns, bit for
bit, alone and inside a batch."""
import numpy as np
import pytest

import paper_2202_03215_gb300 as pb
from paper_2202_03215_gb300 import build as pbuild
from paper_2202_03215_gb300 import workloads as w

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    pbuild.build()


def params():
    return w.config_argon_small(n_e0=20_000, n_i0=20_000).with_(drive=w.DRIVE_RI, I_A=1e-3, R_m=0.01)


def same(a, b):
    sa, sb = a.get_state(), b.get_state()
    return all(np.array_equal(sa[k], sb[k]) for k in sa)


def test_ri_column_is_the_e0_column_at_the_resolved_field():
    p = params()
    r = pb.drive_ri(p)
    a = pb.Column(p)
    b = pb.Column(p.with_(drive=w.DRIVE_E0, E0_Vpm=r["E0_Vpm"], n0_m3=r["n0_m3"]))
    assert same(a, b)
    a.step(12)
    b.step(12)
    assert same(a, b)
    assert a.stats()["births"] == b.stats()["births"]
    a.close()
    b.close()


def test_ri_column_in_a_batch():
    p = params()
    r = pb.drive_ri(p)
    q = p.with_(drive=w.DRIVE_E0, E0_Vpm=r["E0_Vpm"], n0_m3=r["n0_m3"])
    b = pb.Batch([p.with_(column=0), q.with_(column=1, seed=p.seed)])
    lone = pb.Column(q.with_(column=0))
    b.step(6)
    lone.step(6)
    assert same(b.columns[0], lone)
    b.close()
    lone.close()
