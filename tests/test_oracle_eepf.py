"""Pins of the oracle's electron energy histogram (Sec. III.C: the EEPF F(x, eps),
normalised so that int eps^(1/2) F deps = 1): each diagnostic sample holds exactly
the live electrons of the state the step leaves, binned by cell and energy, and the
exact Maxwell-model swarm (constant collision frequency) has a Maxwellian EEPF,
ln F linear in eps with slope -1/kT, kT = (2/3) of the isotropic mean energy."""
import numpy as np
import pytest

import oracle
import paper_2202_03215_gb300 as pb
from paper_2202_03215_gb300 import workloads as w
from tests.helpers import QE, ME, AMU, maxwell_model_xsec, n_gas


def expected_bins(st, N, nx, ne, emax, f32):
    t = np.float32 if f32 else np.float64
    K = t(0.5 * ME / QE)
    vx, vy, vz = (st[k].astype(t) for k in ("vx_e", "vy_e", "vz_e"))
    eps = K * (vx * vx + vy * vy + vz * vz)
    x = eps * t(ne / emax)
    b = np.where(x < t(ne), np.floor(np.where(x < t(ne), x, 0)).astype(np.int64), ne)
    bx = (st["cell_e"].astype(np.int64) * nx) // N
    h = np.zeros((nx, ne + 1), np.uint64)
    np.add.at(h, (bx, b), 1)
    return h


@pytest.mark.parametrize("precision", [w.FP64, w.MIXED])
def test_samples_are_the_states_binned(precision):
    # population held fixed (births only counted), so the state after a step is the sampled one
    p = w.config_argon_small(n_e0=3000, n_i0=3000, precision=precision, diag_every=1, ion_subcycle=1,
                             loss_mode=w.LOSS_SWARM)
    o = oracle.Oracle(p)
    nx, ne, emax = 7, 40, 12.0
    o.eepf_config(nx, ne, emax)
    want = np.zeros((nx, ne + 1), np.uint64)
    for _ in range(6):
        o.step(1)
        want += expected_bins(o.get_state(), p.n_cells, nx, ne, emax, precision == w.MIXED)
    got, ns = o.eepf()
    assert ns == 6
    assert got.sum() == 6 * o.stats()["n_e"]
    assert np.array_equal(got, want)
    assert got[:, -1].sum() > 0          # the tail above eps_max is kept, not dropped
    _, ns0 = o.eepf(reset=True)
    got2, ns2 = o.eepf()
    assert ns2 == 0 and got2.sum() == 0


def test_maxwell_model_eepf_is_maxwellian():
    nu, E0, M_amu, dt = 5e9, 2784.0, 0.1, 2e-11
    xs = [maxwell_model_xsec(nu, n_gas(), 100.0, 8193)]
    p = w.Params(gas_mass_amu=M_amu, L_m=0.01, n_cells=100, dt_s=dt, xsec=xs, eps_max_e_eV=100.0,
                 field_mode=w.FIELD_APPLIED, drive=w.DRIVE_E0, E0_Vpm=E0, n_e0=4000, n_i0=0, ion_subcycle=0,
                 loss_mode=w.LOSS_SWARM, Te0_eV=0.5, seed=6, diag_every=50)
    o = oracle.Oracle(p)
    o.step(5000)
    emax, ne = 60.0, 300
    o.eepf_config(1, ne, emax)
    o.step(20000)
    c, ns = o.eepf()
    assert ns == 400 and c.sum() == 400 * 4000
    assert c[0, -1] < 1e-4 * c.sum()            # 60 eV is far out in the tail
    eps, F = pb.eepf_normalized(c, emax)
    # kT of the exact discrete-time Maxwell model: (2/3) of the mean energy less the drift energy
    a = QE * E0 / ME
    P = 1 - np.exp(-nu * dt)
    em = 2 * ME / (M_amu * AMU)
    q = 1 - P * (1 - em / 6)
    wd = a * dt * q / (P * (1 - em / 6))
    v2 = (1 - P * em) * (2 * a * dt * wd + (a * dt) ** 2) / (P * em)
    kT = 2.0 / 3.0 * 0.5 * ME / QE * (v2 - wd * wd)
    n = c[0, :-1].astype(float)
    k = (eps > 0.3 * kT) & (eps < 5 * kT) & (n > 0)
    slope, icpt = np.polyfit(eps[k], np.log(F[0, k]), 1, w=np.sqrt(n[k]))
    assert slope == pytest.approx(-1.0 / kT, rel=0.03)
    # and the normalisation: sum eps^(1/2) F deps = 1
    assert (F[0] * np.sqrt(eps) * (emax / ne)).sum() == pytest.approx(1.0, rel=1e-12)
