"""Pins of the oracle's (R, I) drive (Sec. II, eq. 2: nu_i = (2.4/R)^2 D_a,
D_a = D_e mu_i / mu_e, and J = e n0 (mu_e + mu_i) E0): the exact similarity laws of
eq. 2, linearity in the current, the scalings of the low-field ion mobility with
temperature and cross section, and parity with the library's host-side drive."""
import numpy as np
import pytest

from oracle import two_term as tt
from paper_2202_03215_gb300 import workloads as w



def neon(**kw):
    return w.config_neon_column(drive=w.DRIVE_RI, I_A=1e-3, R_m=0.01).with_(**kw)


def ri(p):
    xs = [(x.kind, x.threshold_eV, x.energy_eV, x.sigma_m2) for x in p.xsec]
    return tt.ri_drive(xs, p.gas_mass_amu, p.pressure_torr, p.T_gas_K, p.R_m, p.I_A, p.eps_max_e_eV)


def test_similarity_in_pR():
    # at fixed pR, E/N (so E0/p) is the same; J = I/(pi R^2) and mu ~ 1/p make n0 scale as 1/R^2
    E1, n1, m1 = ri(neon())
    E2, n2, m2 = ri(neon(pressure_torr=2.0, R_m=0.005))
    assert E2 / 2.0 == pytest.approx(E1, rel=1e-9)
    assert n2 == pytest.approx(4.0 * n1, rel=1e-9)
    assert m2 == pytest.approx(m1, rel=1e-12)


def test_current_scales_the_density_only():
    E1, n1, _ = ri(neon())
    E2, n2, _ = ri(neon(I_A=5e-3))
    assert E2 == E1
    assert n2 == pytest.approx(5.0 * n1, rel=1e-12)


def test_balance_holds_at_the_root():
    p = neon()
    E0, n0, muN = ri(p)
    N = p.pressure_torr * tt.TORR / (tt.KB * p.T_gas_K)
    xs = [(x.kind, x.threshold_eV, x.energy_eV, x.sigma_m2) for x in p.xsec if x.kind <= 2]
    s = tt.solve(xs, p.gas_mass_amu, E0 / N / tt.TD, eps_max=p.eps_max_e_eV, n=800)
    nu_i = N * s["nu_izN"]
    loss = (muN / N) * (s["DN"] / s["muN"]) * (2.405 / p.R_m) ** 2
    assert nu_i == pytest.approx(loss, rel=1e-8)
    # the current density of eq. 2's column
    J = n0 * tt.QE * (s["muN"] / N + muN / N) * E0
    assert J * np.pi * p.R_m ** 2 == pytest.approx(p.I_A, rel=1e-9)


def test_ion_mobility_scalings():
    e, s = np.array([0.0, 100.0]), np.array([3e-19, 3e-19])
    m = tt.ion_mobility_N([(tt.ION_CX, 0.0, e, s)], w.AMU_NE, 300.0)
    # a charge exchange transfers twice its cross section: as an isotropic process of 2 sigma
    assert tt.ion_mobility_N([(tt.ION_ISO, 0.0, e, 2 * s)], w.AMU_NE, 300.0) == pytest.approx(m, rel=1e-14)
    # constant cross section: mu N ~ (M T)^(-1/2) / Q
    assert tt.ion_mobility_N([(tt.ION_CX, 0.0, e, s)], w.AMU_NE, 1200.0) == pytest.approx(m / 2, rel=1e-14)
    assert tt.ion_mobility_N([(tt.ION_CX, 0.0, e, s)], 4 * w.AMU_NE, 300.0) == pytest.approx(m / 2, rel=1e-14)
    assert tt.ion_mobility_N([(tt.ION_CX, 0.0, e, 3 * s)], w.AMU_NE, 300.0) == pytest.approx(m / 3, rel=1e-14)


def test_parity_with_the_library_drive():
    # host code of the library (pic_drive_ri): its own two-term scheme and bisection
    import paper_2202_03215_gb300 as pb
    from paper_2202_03215_gb300 import build as pbuild
    pbuild.build()
    for kw in ({}, {"pressure_torr": 0.5, "R_m": 0.02, "I_A": 5e-3}):
        p = neon(**kw)
        E0, n0, muN = ri(p)
        r = pb.drive_ri(p)
        assert r["E0_Vpm"] == pytest.approx(E0, rel=1e-5)
        assert r["n0_m3"] == pytest.approx(n0, rel=1e-5)
        assert r["mu_iN"] == pytest.approx(muN, rel=1e-12)
