"""The library's two-term transport (pic_two_term: exponential flux scheme,
Hessenberg elimination; host code, no GPU) against the oracle's independent
solve (central differences, dense solve) and the Maxwell-model closed forms."""
import numpy as np
import pytest

import paper_2202_03215_gb300 as pb
from paper_2202_03215_gb300 import build as pbuild
from paper_2202_03215_gb300 import workloads as w
from oracle import two_term as tt

KEYS = [("mean_eps", "mean_eps_eV"), ("muN", "muN"), ("DN", "DN"), ("mueN", "mueN"), ("DeN", "DeN"),
        ("loss_N", "lossN"), ("power_N", "powerN")]


@pytest.fixture(scope="module", autouse=True)
def _built():
    pbuild.build()


@pytest.mark.parametrize("gas", ["neon", "argon"])
def test_two_term_matches_oracle(gas):
    xs = w.neon_xsecs() if gas == "neon" else w.argon_xsecs()
    mass = w.AMU_NE if gas == "neon" else w.AMU_AR
    xo = [(x.kind, x.threshold_eV, x.energy_eV, x.sigma_m2) for x in xs if x.kind <= 2]
    ens = [3.0, 10.0, 30.0, 100.0]
    got = pb.two_term(xs, mass, ens, eps_max_eV=120.0, n_grid=1000)
    for en, g in zip(ens, got):
        o = tt.solve(xo, mass, en, eps_max=120.0, n=2000)
        for ko, kg in KEYS:
            assert g[kg] == pytest.approx(o[ko], rel=1e-2), (gas, en, kg)
        if en >= 10.0:    # ionization well resolved (not only the far tail)
            assert g["nu_izN"] == pytest.approx(o["nu_izN"], rel=2e-2), (gas, en)
        assert g["alphaN"] == pytest.approx(g["nu_izN"] / (g["muN"] * en * 1e-21), rel=1e-12)


def test_two_term_maxwell_model():
    N, nu = 3.219e22, 2e9
    e = np.concatenate([[0.0], np.geomspace(1e-6, 1000.0, 4000)])
    s = nu / (N * tt.GAMMA * np.sqrt(np.maximum(e, 1e-12)))
    s[0] = s[1]
    xs = [w.XSec(w.ELASTIC, e, s)]
    vd = tt.QE * 1e-21 * N / (tt.ME * nu)
    kT = w.AMU_NE * tt.AMU * vd ** 2 / (3 * tt.QE)
    g = pb.two_term(xs, w.AMU_NE, [1.0], eps_max_eV=40 * kT, n_grid=2000)[0]
    assert g["mean_eps_eV"] == pytest.approx(1.5 * kT, rel=1e-3)
    assert g["muN"] / N == pytest.approx(tt.QE / (tt.ME * nu), rel=1e-3)
    assert g["DN"] / g["muN"] == pytest.approx(kT, rel=1e-3)
    assert g["mueN"] / g["muN"] == pytest.approx(5 / 3, rel=1e-3)
    assert g["DeN"] / g["DN"] == pytest.approx(5 / 3, rel=1e-3)


def test_two_term_rejects_bad_arguments():
    with pytest.raises(pb.PicError):
        pb.two_term(w.neon_xsecs(), w.AMU_NE, [-1.0])
    with pytest.raises(pb.PicError):
        pb.two_term(w.neon_xsecs(), w.AMU_NE, [10.0], n_grid=10)


def test_multilevel_transport_matches_the_oracle():
    from paper_2202_03215_gb300 import workloads as w
    xs = [x for x in w.neon_multilevel_xsecs() if x.kind <= 2]
    xo = [(x.kind, x.threshold_eV, x.energy_eV, x.sigma_m2) for x in xs]
    for en in (30.0, 80.0):
        g = pb.two_term(xs, w.AMU_NE, [en], eps_max_eV=200.0, n_grid=1000)[0]
        o = tt.solve(xo, w.AMU_NE, en, eps_max=200.0, n=1000)
        for kg, ko in (("mean_eps_eV", "mean_eps"), ("muN", "muN"), ("nu_izN", "nu_izN")):
            assert g[kg] == pytest.approx(o[ko], rel=1e-4), (en, kg)

