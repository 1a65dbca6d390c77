"""Uniform-field electron swarms run by the GPU particle step (field applied,
ionizations counted, population held fixed) against the oracle's independent
two-term Boltzmann solve (Sec. III.B: uniform-field PIC-MCC reproduces the
Boltzmann-solver swarm data).  Bands: 5% on the drift velocity and the mean
energy, 15% on the ionization coefficient alpha = nu_iz / w (the two-term
approximation loses accuracy as inelastic collisions take over)."""
import numpy as np
import pytest

from oracle import two_term as tt
from paper_2202_03215_gb300 import build as pbuild
from paper_2202_03215_gb300 import closure as cl
from paper_2202_03215_gb300 import workloads as w

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    pbuild.build()


def test_swarm_matches_two_term():
    ens = [10.0, 30.0, 100.0]
    xo = [(x.kind, x.threshold_eV, x.energy_eV, x.sigma_m2) for x in w.neon_xsecs() if x.kind <= 2]
    ref = [tt.solve(xo, w.AMU_NE, en, eps_max=150.0, n=1500) for en in ens]
    ps = [cl.swarm_params(en, n=50_000, column=k).with_(dt_s=2e-11, Te0_eV=r["Te"])
          for k, (en, r) in enumerate(zip(ens, ref))]
    mom, births = cl.run_windows(ps, 20_000, 4, 2500)
    for en, p, ms, nb, r in zip(ens, ps, mom, births, ref):
        ne = sum(m["n_e"].sum() for m in ms)
        wd = sum(m["gamma_e"].sum() for m in ms) / ne
        eps = sum((m["mean_eps_e"] * m["n_e"]).sum() for m in ms) / ne
        eps_iso = eps - 0.5 * tt.ME * wd * wd / tt.QE     # drift energy is beyond the two-term F0
        nu = nb / (p.n_e0 * 4 * 2500 * p.dt_s)
        N = cl.n_gas(p)
        assert wd == pytest.approx(r["drift"], rel=0.05), en
        assert eps_iso == pytest.approx(r["mean_eps"], rel=0.05), en
        if en >= 30.0:     # >= 5000 ionizations in the window
            assert nu / wd / N == pytest.approx(r["alphaN"], rel=0.15), en
