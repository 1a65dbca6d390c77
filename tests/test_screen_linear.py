"""Pins of the linear-stability screen (Sec. IV.B, eqs. 18-23, and the full linearisation of the fluid
model) on a synthetic transport table where the answer is known in closed form: transport
coefficients independent of Te and an ionization frequency with no Te dependence (nu_i' = 0).
Then the density perturbation decouples from the temperature: it decays by ambipolar diffusion,
gamma = -a0 D k^2 with a0 = mu_i/(mu_e + mu_i), and does not move (omega = 0); the energy
perturbation decays by heat conduction and the loss slope, gamma = -D_eps k^2 - (2/3) dL/dTe,
and drifts with the energy mobility, omega = -k mu_eps E0.  Eq. (19)'s growth rate reduces to
-D_a k^2 with D_a = D_e mu_i / mu_e (eq. 2)."""
import math

import numpy as np
import pytest

from paper_2202_03215_gb300 import screen

N_GAS = 3.2e22
MU_N, D_N, MUE_N, DE_N = 1.0e24, 3.0e24, 1.67e24, 5.0e24
MU_I = 0.05
T0, N0, E0 = 2.0, 1e15, 500.0


def _table(loss_slope_N):
    Te = np.array([0.5, 1.0, 2.0, 3.0, 4.0])
    recs = [dict(mean_eps_eV=1.5 * t, muN=MU_N, DN=D_N, mueN=MUE_N, DeN=DE_N, nu_izN=1e-14,
                 lossN=1e-13 + loss_slope_N * t) for t in Te]
    return screen.Table(recs)


def _state():
    mu = MU_N / N_GAS
    return screen.Homogeneous(p_torr=1.0, N_gas=N_GAS, T0=T0, E0=E0, nu_w=1e-14 * N_GAS, n0=N0,
                              Gamma_T=N0 * (mu + MU_I) * E0, mu_e=mu, mu_i=MU_I, D_e=D_N / N_GAS)


@pytest.mark.parametrize("k", [50.0, 200.0, 800.0])
def test_density_mode_is_ambipolar_diffusion(k):
    tab, h = _table(loss_slope_N=4e-14), _state()    # a strongly damped energy mode
    g, om, v = screen.dispersion(tab, h, k, vector=True)
    mu, D = MU_N / N_GAS, D_N / N_GAS
    assert g == pytest.approx(-MU_I / (mu + MU_I) * D * k * k, rel=1e-9)
    assert abs(om) <= 1e-9 * abs(g)
    assert abs(v[1]) <= 1e-9 * abs(v[0])              # a pure density perturbation


@pytest.mark.parametrize("k", [50.0, 200.0])
def test_energy_mode_when_it_is_the_least_damped(k):
    # a loss falling steeply with Te: the energy mode grows, the density mode decays
    slope = -3e-14
    tab, h = _table(loss_slope_N=slope), _state()
    g, om = screen.dispersion(tab, h, k)
    De, mue = DE_N / N_GAS, MUE_N / N_GAS
    assert g == pytest.approx(-De * k * k - 2.0 / 3.0 * slope * N_GAS, rel=1e-6)
    assert om == pytest.approx(-k * mue * E0, rel=1e-9)


def test_eq19_growth_rate_reduces_to_ambipolar_diffusion():
    tab, h = _table(loss_slope_N=4e-14), _state()
    Da = h.mu_i * (D_N / N_GAS) / (MU_N / N_GAS)
    for k in (50.0, 200.0):
        g, om = screen.gamma_k(tab, h, k)
        assert g == pytest.approx(-Da * k * k, rel=1e-9)
        assert om == 0.0
    lin = screen.linear(tab, h)
    assert lin["nu_p"] == 0.0 and not lin["unstable"]


def test_closed_form_maximum_is_the_maximum_of_eq19():
    """eqs. (21)-(22) give the fastest-growing wave number and its growth rate in closed form;
    a direct search of eq. (19)'s gamma(k) over k must find the same maximum, and the phase
    velocity is omega(k_max)/k_max."""
    from scipy.optimize import minimize_scalar
    tab = screen.Table(screen.transport())
    found = 0
    for E0p in (6.0, 8.0, 12.0, 16.0):
        h = screen.homogeneous_E0(tab, E0p, 1.0)
        lin = screen.linear(tab, h)
        if not lin["unstable"]:
            continue
        found += 1
        ks = np.geomspace(lin["k_max"] / 30, lin["k_max"] * 30, 400)
        g = np.array([screen.gamma_k(tab, h, k)[0] for k in ks])
        i = int(np.argmax(g))
        assert 0 < i < len(ks) - 1                       # an interior maximum
        r = minimize_scalar(lambda lk: -screen.gamma_k(tab, h, math.exp(lk))[0],
                            bracket=(math.log(ks[i - 1]), math.log(ks[i]), math.log(ks[i + 1])), tol=1e-10)
        k_best = math.exp(r.x)
        assert k_best == pytest.approx(lin["k_max"], rel=1e-4)
        assert -r.fun == pytest.approx(lin["gamma_max"], rel=1e-8)
        g_at, om_at = screen.gamma_k(tab, h, lin["k_max"])
        assert om_at / lin["k_max"] == pytest.approx(lin["v_ph"], rel=1e-12)
        assert lin["lam"] == pytest.approx(2 * math.pi / lin["k_max"], rel=1e-12)
    assert found >= 2
