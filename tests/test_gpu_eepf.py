"""The electron energy histogram on the GPU (pic_eepf_*; Sec. III.C, the EEPF
F(x, eps)): bit-exact against the oracle's histogram over steps with births,
removals and ion steps, in both storage forms; and, for a uniform-field neon
swarm, the normalised EEPF against the oracle's two-term solution F0 (the
paper's Fig. 8 comparison of uniform-field PIC-MCC with a Boltzmann solver)."""
import numpy as np
import pytest

import oracle
import paper_2202_03215_gb300 as pb
from oracle import two_term as tt
from paper_2202_03215_gb300 import build as pbuild
from paper_2202_03215_gb300 import closure as cl
from paper_2202_03215_gb300 import workloads as w

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    pbuild.build()


@pytest.mark.parametrize("precision", [w.FP64, w.MIXED])
def test_histogram_matches_the_oracle(precision):
    p = w.config_argon_small(n_e0=20_000, n_i0=20_000, precision=precision, diag_every=10)
    g, o = pb.Column(p), oracle.Oracle(p)
    for h in (g, o):
        h.eepf_config(25, 64, 30.0)
    g.step(40)
    o.step(40)
    cg, ng = g.eepf()
    co, no = o.eepf()
    assert ng == no == 4
    assert cg.sum() == 4 * g.stats()["n_e"]
    assert np.array_equal(cg, co)
    assert g.stats()["births"] == o.stats()["births"] > 0
    cg2, ng2 = g.eepf(reset=True)
    assert np.array_equal(cg2, cg)
    cg3, ng3 = g.eepf()
    assert ng3 == 0 and cg3.sum() == 0
    g.close()


def test_histogram_rejects_bad_shapes_and_batches():
    p = w.config_argon_small(n_e0=2000, n_i0=2000, diag_every=10)
    g = pb.Column(p)
    for bad in ((0 - 1, 10, 5.0), (p.n_cells + 1, 10, 5.0), (4, 0, 5.0), (4, 10, 0.0)):
        with pytest.raises(pb.PicError):
            g.eepf_config(*bad)
    with pytest.raises(pb.PicError):
        g._eepf_shape = (1, 1)
        g.eepf()                          # not configured
    g.close()
    b = pb.Batch([p, p.with_(seed=2)])
    with pytest.raises(pb.PicError):
        b.columns[0].eepf_config(4, 10, 5.0)
    b.close()


def test_uniform_field_swarm_eepf_against_two_term():
    EN = 30.0
    xo = [(x.kind, x.threshold_eV, x.energy_eV, x.sigma_m2) for x in w.neon_xsecs() if x.kind <= 2]
    ref = tt.solve(xo, w.AMU_NE, EN, eps_max=150.0, n=1500)
    p = cl.swarm_params(EN, n=100_000).with_(dt_s=2e-11, Te0_eV=ref["Te"])
    g = pb.Column(p)
    g.step(20_000)                        # relaxed
    emax, ne = 40.0, 80
    g.eepf_config(1, ne, emax)
    g.step(20_000)
    c, ns = g.eepf()
    assert ns == 20_000 // p.diag_every
    eps, F = pb.eepf_normalized(c, emax)
    F0 = np.interp(eps, ref["eps"], ref["F"])
    # the bulk and the inelastic knee: within 15 % where the two-term F0 is above 1e-3 of its peak
    k = (eps > 1.0) & (F0 > 1e-3 * F0.max())
    assert np.max(np.abs(F[0, k] / F0[k] - 1)) < 0.15
    g.close()
