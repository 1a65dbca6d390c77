"""Pins of the oracle's two-term Boltzmann solve (the fluid-model closure source,
Sec. IV.A, eqs. 6-9) against closed forms of the two-term equation."""
import math

import numpy as np
import pytest

from oracle import two_term as tt
from paper_2202_03215_gb300 import workloads as w

N_GAS = 3.219e22
NU = 2e9


def maxwell_sigma():
    """sigma(eps) with constant collision frequency NU at gas density N_GAS."""
    e = np.concatenate([[0.0], np.geomspace(1e-6, 1000.0, 4000)])
    s = NU / (N_GAS * tt.GAMMA * np.sqrt(np.maximum(e, 1e-12)))
    s[0] = s[1]
    return e, s


@pytest.mark.parametrize("EN_Td", [0.5, 1.0])
def test_maxwell_model(EN_Td):
    # constant nu_m, elastic only: F is Maxwellian with kT = M v_d^2 / 3, v_d = eE/(m nu);
    # mu = e/(m nu), D = kT mu, mu_eps = 5/3 mu, D_eps = 5/3 D (all exact)
    e, s = maxwell_sigma()
    M = w.AMU_NE
    E = EN_Td * tt.TD * N_GAS
    vd = tt.QE * E / (tt.ME * NU)
    kT = M * tt.AMU * vd ** 2 / (3 * tt.QE)
    r = tt.solve([(tt.ELASTIC, 0.0, e, s)], M, EN_Td, eps_max=40 * kT, n=2000)
    assert r["mean_eps"] == pytest.approx(1.5 * kT, rel=1e-3)
    assert r["drift"] == pytest.approx(vd, rel=1e-3)
    assert r["muN"] / N_GAS == pytest.approx(tt.QE / (tt.ME * NU), rel=1e-3)
    assert r["DN"] / r["muN"] == pytest.approx(kT, rel=1e-3)
    assert r["mueN"] / r["muN"] == pytest.approx(5.0 / 3.0, rel=1e-3)
    assert r["DeN"] / r["DN"] == pytest.approx(5.0 / 3.0, rel=1e-3)
    # Maxwellian shape: ln F linear in eps with slope -1/kT over the bulk
    k = (r["eps"] > 0.2 * kT) & (r["eps"] < 8 * kT)
    slope = np.polyfit(r["eps"][k], np.log(r["F"][k]), 1)[0]
    assert slope == pytest.approx(-1.0 / kT, rel=2e-3)


@pytest.mark.parametrize("EN_Td", [5.0, 20.0])
def test_druyvesteyn(EN_Td):
    # constant sigma, elastic only: F ~ exp(-(eps/eD)^2), eD^2 = (E/N)^2 M / (3 m sigma^2);
    # mean energy eD G(5/4)/G(3/4); mu N = gamma/(3 sigma) sqrt(pi) / (eD^(1/2) G(3/4))
    s0 = 2e-20
    M = w.AMU_NE
    EN = EN_Td * tt.TD
    eD = math.sqrt(EN ** 2 * M * tt.AMU / (3 * tt.ME * s0 ** 2))
    r = tt.solve([(tt.ELASTIC, 0.0, np.array([0.0, 1e3]), np.array([s0, s0]))], M, EN_Td,
                 eps_max=5 * eD, n=2000)
    assert r["mean_eps"] == pytest.approx(eD * math.gamma(1.25) / math.gamma(0.75), rel=1e-3)
    muN = tt.GAMMA / (3 * s0) * math.sqrt(math.pi) / (math.sqrt(eD) * math.gamma(0.75))
    assert r["muN"] == pytest.approx(muN, rel=1e-3)


def test_excitation_absorber():
    # Maxwell-model heating, no elastic cooling (very heavy gas), a strong excitation
    # above u: electrons reaching u are returned to ~0, the flux below u is constant and
    # F = C (eps^-1/2 - u^-1/2) -> mean energy 0.3 u (exact as the absorber becomes
    # perfect; the finite penetration depth adds < 1%); the heating power equals u nu_exc.
    e, s = maxwell_sigma()
    u = 10.0
    exc = (tt.EXCITATION, u, np.array([u, 1000.0]), np.array([3e-20, 3e-20]))
    r = tt.solve([(tt.ELASTIC, 0.0, e, s), exc], 1e6, 1.0, eps_max=12.0, n=2000)
    assert r["mean_eps"] == pytest.approx(0.3 * u, rel=1e-2)
    assert r["mean_eps"] > 0.3 * u
    assert r["power_N"] == pytest.approx(u * r["nuN"][1], rel=1e-3)


def neon_electron_xsecs():
    return [(x.kind, x.threshold_eV, x.energy_eV, x.sigma_m2) for x in w.neon_xsecs() if x.kind <= 2]


@pytest.mark.parametrize("EN_Td", [10.0, 30.0, 100.0])
def test_neon_energy_balance_and_convergence(EN_Td):
    # steady state: power gained from the field = elastic + inelastic losses, with the
    # ionization loss of the swarm mode (the scattered electron keeps a uniform share)
    xs = neon_electron_xsecs()
    r = tt.solve(xs, w.AMU_NE, EN_Td, eps_max=120.0, n=2000)
    assert r["power_N"] == pytest.approx(r["swarm_loss_N"], rel=1e-4)
    assert r["F"].min() > -1e-12 * r["F"].max()
    r2 = tt.solve(xs, w.AMU_NE, EN_Td, eps_max=120.0, n=1000)
    for k in ("mean_eps", "muN", "DN", "mueN", "DeN"):
        assert r2[k] == pytest.approx(r[k], rel=1e-2)
    assert r2["nu_izN"] == pytest.approx(r["nu_izN"], rel=3e-2)


def test_neon_trends():
    xs = neon_electron_xsecs()
    rs = [tt.solve(xs, w.AMU_NE, en, eps_max=120.0, n=1000) for en in (3.0, 10.0, 30.0, 100.0)]
    eb = [r["mean_eps"] for r in rs]
    wd = [r["drift"] for r in rs]
    al = [r["alphaN"] for r in rs]
    assert np.all(np.diff(eb) > 0) and np.all(np.diff(wd) > 0) and np.all(np.diff(al) > 0)
