"""The (R, I) drive (Sec. II, eq. 2): pic_drive_ri (host code, no GPU) against an
independent bisection on the oracle's two-term solve, and the exact similarity
laws of eq. 2: E0/p depends on pR only, n0 scales with I/R at fixed pR."""
import math

import numpy as np
import pytest

import paper_2202_03215_gb300 as pb
from oracle import two_term as tt
from paper_2202_03215_gb300 import build as pbuild
from paper_2202_03215_gb300 import workloads as w

KB, TORR = 1.380649e-23, 133.32236842105263


@pytest.fixture(scope="module", autouse=True)
def _built():
    pbuild.build()


def neon(**kw):
    return w.config_neon_column(drive=w.DRIVE_RI, I_A=1e-3, R_m=0.01, **kw)


def test_root_and_density_against_the_oracle_two_term():
    p = neon()
    r = pb.drive_ri(p)
    N = p.pressure_torr * TORR / (KB * p.T_gas_K)
    mu_i = r["mu_iN"] / N
    g2 = (2.405 / p.R_m) ** 2
    xo = [(x.kind, x.threshold_eV, x.energy_eV, x.sigma_m2) for x in p.xsec if x.kind <= 2]

    def f(EN):
        s = tt.solve(xo, p.gas_mass_amu, EN, eps_max=p.eps_max_e_eV, n=1000)
        return N * s["nu_izN"] - mu_i * (s["DN"] / s["muN"]) * g2, s

    lo, hi = math.log(5.0), math.log(100.0)
    assert f(math.exp(lo))[0] < 0 < f(math.exp(hi))[0]
    for _ in range(30):
        mid = 0.5 * (lo + hi)
        if f(math.exp(mid))[0] < 0:
            lo = mid
        else:
            hi = mid
    EN = math.exp(0.5 * (lo + hi))
    _, s = f(EN)
    E0 = EN * 1e-21 * N
    J = p.I_A / (math.pi * p.R_m ** 2)
    n0 = J / (tt.QE * (s["muN"] / N + mu_i) * E0)
    assert r["E0_Vpm"] == pytest.approx(E0, rel=0.02)
    assert r["n0_m3"] == pytest.approx(n0, rel=0.03)
    assert r["Te0_eV"] == pytest.approx(s["Te"], rel=0.02)


def test_ion_mobility_near_the_particle_models_ion_drift():
    # uniform-phase ion drift of the particle model's neon columns at 18.6 Td: mu_i N = 1.39e22
    assert pb.drive_ri(neon())["mu_iN"] == pytest.approx(1.39e22, rel=0.15)


def test_similarity_laws_of_eq_2():
    a = pb.drive_ri(neon())
    b = pb.drive_ri(neon().with_(pressure_torr=2.0, R_m=0.005))           # same pR, same I
    c = pb.drive_ri(neon().with_(pressure_torr=2.0, R_m=0.005, I_A=5e-4))  # same pR, same I/R
    assert b["E0_Vpm"] / 2.0 == pytest.approx(a["E0_Vpm"], rel=1e-8)
    assert b["n0_m3"] == pytest.approx(4 * a["n0_m3"], rel=1e-8)
    assert c["n0_m3"] == pytest.approx(2 * a["n0_m3"], rel=1e-8)
    assert b["Te0_eV"] == pytest.approx(a["Te0_eV"], rel=1e-8)
    d = pb.drive_ri(neon().with_(I_A=2e-3))                                # n0 linear in I
    assert d["n0_m3"] == pytest.approx(2 * a["n0_m3"], rel=1e-12)
    assert d["E0_Vpm"] == pytest.approx(a["E0_Vpm"], rel=1e-12)


def test_bad_arguments():
    with pytest.raises(pb.PicError):
        pb.drive_ri(neon().with_(R_m=0.0))
    with pytest.raises(pb.PicError):
        pb.drive_ri(neon().with_(xsec=[x for x in w.neon_xsecs() if x.kind <= 2]))   # no ion process
