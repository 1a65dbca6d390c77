"""The fluid screen on the GPU: linearity in density (Sec. II / T10: the current
only scales n0, so a column at 4x the current is the same column scaled by 4,
bit for bit in FP32 because 4 is a power of two) and the linear phase of an
ionization wave against the full linearisation of the fluid equations."""
import math

import numpy as np
import pytest

import paper_2202_03215_gb300 as pb
from paper_2202_03215_gb300 import build as pbuild
from paper_2202_03215_gb300 import screen as sc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    pbuild.build()


@pytest.fixture(scope="module")
def records():
    return sc.transport()


def test_current_only_scales_the_density(records):
    tab = sc.Table(records)
    h1 = sc.homogeneous_R(tab, 0.5, 0.05)
    h4 = sc.homogeneous_R(tab, 0.5, 0.2)
    assert h4.Gamma_T == pytest.approx(4 * h1.Gamma_T, rel=1e-12)
    h4.Gamma_T = 4 * h1.Gamma_T        # exactly 4x in binary
    cols = sc.fluid_columns([h1, h4], 0.3, 1024)
    f = pb.Fluid(cols, records, n_T=128, dt_s=2e-8, diag_every=50, n_modes=16)
    n, T = sc.initial_state(1024, h1, 5)
    f.set_state(0, n, T)
    f.set_state(1, 4 * n, T)
    f.step(500)
    n1, T1 = f.get_state(0)
    n4, T4 = f.get_state(1)
    assert np.array_equal(n4, 4 * n1)
    assert np.array_equal(T4, T1)
    rec = f.modes()
    assert np.array_equal(rec[:, 1], 4 * rec[:, 0])
    f.close()


@pytest.mark.parametrize("E0p,m", [(8.0, 10), (12.0, 12), (16.0, 16)])
def test_linear_phase_against_the_dispersion_relation(records, E0p, m):
    # a single small mode grows and travels as the full linearisation of eqs. 3-5, 8-9, 11, 17
    # predicts (growth rate and phase velocity within 15 %: the grid and time step of the
    # integration against the continuum; dt is small against the damped energy root, whose
    # rate |Omega| ~ 3e8 /s sets the splitting error); the paper's eq. (20) agrees on the sign
    tab = sc.Table.uniform(records, 128)          # the kernel's own table (its slopes enter omega)
    h = sc.homogeneous_E0(tab, E0p, 1.0)
    L = 0.10
    k = 2 * math.pi * m / L
    g_lin, om_lin, vec = sc.dispersion(tab, h, k, vector=True)
    assert g_lin > 0 and sc.gamma_k(tab, h, k)[0] > 0
    N = 2048
    cols = sc.fluid_columns([h], L, N, pair=False)
    dt = 5e-10
    steps = int(round(4.0 / g_lin / dt))
    de = max(1, steps // 60)
    f = pb.Fluid(cols, records, n_T=128, dt_s=dt, diag_every=de, n_modes=m)
    x = np.arange(N) / N
    # the growing eigenmode: dn = 1e-5 n0, dT = (v_T / v_n) dn
    dn = 1e-5 * h.n0
    dT = vec[1] / vec[0] * dn
    ph = np.exp(2j * math.pi * m * x)
    f.set_state(0, h.n0 + (dn * ph).real, h.T0 + (dT * ph).real)
    f.step(steps)
    rec = f.modes()[:, 0]
    f.close()
    t = (np.arange(len(rec)) + 1) * de * dt
    amp = np.abs(rec[:, m])
    sel = t > 1.0 / g_lin                 # after the transient of the temperature response
    gam = np.polyfit(t[sel], np.log(amp[sel]), 1)[0]
    ph = np.unwrap(np.angle(rec[sel, m]))
    v = -np.polyfit(t[sel], ph, 1)[0] / k
    assert gam == pytest.approx(g_lin, rel=0.15)
    assert v == pytest.approx(om_lin / k, rel=0.15)
