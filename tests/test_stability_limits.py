"""pic_check_stability (host only, no GPU): the resolution limits of the explicit
particle scheme that Sec. II states, dt < 0.2 / w_pe and dx < lambda_De, at the
initial density and electron temperature, against their closed forms."""
import numpy as np
import pytest

import paper_2202_03215_gb300 as pb
from paper_2202_03215_gb300 import build as pbuild
from paper_2202_03215_gb300 import workloads as w
from tests.helpers import EPS0, ME, QE


@pytest.fixture(scope="module", autouse=True)
def _built():
    pbuild.build()


def _closed_form(p):
    wpe = np.sqrt(p.n0_m3 * QE * QE / (EPS0 * ME))
    lde = np.sqrt(EPS0 * p.Te0_eV / (p.n0_m3 * QE))
    return wpe * p.dt_s, (p.L_m / p.n_cells) / lde


def test_argon_parity_column_meets_both_limits():
    p = w.config_argon_small()
    r = pb.check_stability(p)
    a, b = _closed_form(p)
    # w_pe(1e15 m^-3) = 1.78e9 /s, lambda_De(1e15, 2 eV) = 0.33 mm
    assert r["wpe_dt"] == pytest.approx(a, rel=1e-12) and abs(a - 1.784e9 * 2e-11) < 1e-4
    assert r["dx_over_lambda_De"] == pytest.approx(b, rel=1e-12) and abs(b - 1e-4 / 3.325e-4) < 1e-3
    assert r["warnings"] == 0


@pytest.mark.parametrize("kw, bits", [
    (dict(dt_s=1.2e-10), pb.WARN_PLASMA_FREQ),                  # w_pe dt = 0.21
    (dict(n_cells=150), pb.WARN_DEBYE),                          # dx = 0.33 mm = 1.0 lambda_De
    (dict(n0_m3=4e16, n_cells=200), pb.WARN_PLASMA_FREQ | pb.WARN_DEBYE),
    (dict(Te0_eV=0.0), pb.WARN_DEBYE),                           # a cold start resolves no Debye length
])
def test_each_limit_is_reported(kw, bits):
    p = w.config_argon_small(**kw)
    r = pb.check_stability(p)
    assert r["warnings"] == bits, r
    if p.Te0_eV > 0:
        a, b = _closed_form(p)
        assert r["wpe_dt"] == pytest.approx(a, rel=1e-12) and r["dx_over_lambda_De"] == pytest.approx(b, rel=1e-12)


def test_neon_column_with_the_current_drive_uses_the_density_of_eq_2():
    p = w.config_neon_column(n_per_species=1000, drive=w.DRIVE_RI, I_A=1e-3)
    d = pb.drive_ri(p)
    r = pb.check_stability(p)
    a, b = _closed_form(p.with_(n0_m3=d["n0_m3"], Te0_eV=p.Te0_eV))
    assert r["wpe_dt"] == pytest.approx(a, rel=1e-9) and r["dx_over_lambda_De"] == pytest.approx(b, rel=1e-9)
    assert r["warnings"] == 0


def test_invalid_statement_is_an_error():
    with pytest.raises(pb.PicError):
        pb.check_stability(w.config_argon_small(dt_s=-1.0))
