"""The bounded column of Sec. V on the GPU (PIC_FLAG_BOUNDED: absorbing cathode and
anode, Dirichlet field, cathode emission, resistor circuit, fixed loss frequency):
bit-exact against the oracle step by step (particles, node charges, field, absorbed
and emitted counts), the Child-Langmuir current of a vacuum diode, and the
parameter checks."""
import numpy as np
import pytest

import oracle
import paper_2202_03215_gb300 as pb
from paper_2202_03215_gb300 import build as pbuild
from paper_2202_03215_gb300 import workloads as w
from tests.test_oracle_bounded import diode, EPS0
from tests.helpers import QE, ME

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    pbuild.build()


def bounded(precision, drive):
    p = w.config_argon_small(n_e0=20_000, n_i0=20_000, precision=precision, flags=w.FLAG_BOUNDED,
                             loss_mode=w.LOSS_RADIAL, nu_w=1e6, J_emit_Am2=10.0, T_emit_eV=0.5, diag_every=10)
    if drive == "circuit":
        p = p.with_(drive=w.DRIVE_CIRCUIT, U_src=30.0, R_ext_ohm_m2=10.0)
    return p


def same(g, o, where):
    a, b = g.get_state(), o.get_state()
    for k in a:
        if isinstance(a[k], np.ndarray):
            assert np.array_equal(a[k], b[k]), (where, k)
        else:
            assert a[k] == b[k], (where, k)


@pytest.mark.parametrize("precision,drive", [(w.FP64, "voltage"), (w.MIXED, "voltage"), (w.MIXED, "circuit")])
def test_bounded_column_matches_the_oracle(precision, drive):
    p = bounded(precision, drive)
    g, o = pb.Column(p), oracle.Oracle(p)
    same(g, o, "init")
    assert len(g.get_state()["Q_e"]) == p.n_cells + 1
    for k in range(4):
        g.step(10)
        o.step(10)
        same(g, o, f"step {10 * (k + 1)}")
    sg, so = g.stats(), o.stats()
    for key in ("absorbed_e", "absorbed_i", "emitted", "births", "losses_e", "losses_i", "n_e", "n_i"):
        assert sg[key] == so[key], key
    assert sum(sg["absorbed_e"]) > 0 and sg["emitted"] > 0
    mg, mo = g.moments(), o.moments()
    for key in ("n_e", "n_i", "E", "phi"):
        assert np.allclose(mg[key], mo[key], rtol=1e-9, atol=1e-9 * np.abs(mo[key]).max()), key
    g.close()


def test_vacuum_diode_child_langmuir():
    V, d = 100.0, 0.01
    Jcl = 4 * EPS0 / 9 * np.sqrt(2 * QE / ME) * V ** 1.5 / d ** 2
    p = diode(4 * Jcl, V).with_(precision=w.MIXED)
    g = pb.Column(p)
    g.step(4000)
    a0 = g.stats()["absorbed_e"][1]
    g.step(8000)
    wgt = p.n0_m3 * p.L_m / p.n_e0
    J = (g.stats()["absorbed_e"][1] - a0) * QE * wgt / (8000 * p.dt_s)
    assert J == pytest.approx(Jcl, rel=0.08)
    g.close()


def test_bounded_parameter_checks():
    p = bounded(w.MIXED, "voltage")
    with pytest.raises(pb.PicError):
        pb.Column(p.with_(loss_mode=w.LOSS_PAIR))
    with pytest.raises(pb.PicError):
        pb.Column(p.with_(J_emit_Am2=-1.0))
    with pytest.raises(pb.PicError):
        pb.Batch([p, p.with_(seed=2)])
