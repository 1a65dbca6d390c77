"""Host-side preparation of the closure network's training data: the residual
targets are zero on a state whose moments are exactly the tabulated closure,
and the closure evaluated on data agrees with the oracle's fluid step
formulas (eqs. 11, 17, 8-9).  No GPU."""
import numpy as np
import pytest

from oracle import fluid as fl
from paper_2202_03215_gb300 import closure as cl
from paper_2202_03215_gb300 import screen as sc
from paper_2202_03215_gb300 import workloads as w


def uniform_records(nT=64):
    # smooth synthetic transport on a uniform Te grid (both interpolations then coincide)
    out = []
    for k in range(nT):
        Te = 2.0 + 10.0 * k / (nT - 1)
        out.append(dict(mean_eps_eV=1.5 * Te, muN=1e25 * (1 + 0.05 * Te), DN=3e25 * Te, mueN=1.5e25 * (1 + 0.04 * Te),
                        DeN=4e25 * Te, nu_izN=1e-18 * np.exp(-30.0 / Te), lossN=2e-15 * Te ** 1.5))
    return out


def state(N=256, seed=0):
    rng = np.random.default_rng(seed)
    x = np.arange(N) / N
    n = 1e15 * (1 + 0.3 * np.sin(2 * np.pi * 4 * x) + 0.02 * rng.standard_normal(N))
    T = 5.0 + 1.0 * np.cos(2 * np.pi * 4 * x + 0.3)
    return n, T


def test_mirror_is_an_involution():
    rng = np.random.default_rng(1)
    m = {k: rng.standard_normal(16) for k in ("n_e", "gamma_e", "E", "mean_eps_e")}
    m["n_samples"] = 3
    mm = cl.mirror(cl.mirror(m))
    for k in ("n_e", "gamma_e", "E", "mean_eps_e"):
        assert np.array_equal(mm[k], m[k])
    f = cl.mirror(m)
    assert f["n_e"][0] == m["n_e"][0] and f["n_e"][1] == m["n_e"][-1]
    assert f["gamma_e"][1] == -m["gamma_e"][-1]


def test_table_closure_matches_oracle_fluid_formulas():
    recs = uniform_records()
    tab = sc.Table(recs)
    otab = fl.make_table(recs, len(recs))
    n, T = state()
    L, Ng, muiN, GT = 0.1, 3.2e22, 1.3e22, 2e19
    G, H, nu, E = cl.table_closure(n, T, GT, L, Ng, muiN, tab)
    col = dict(L_m=L, N_gas=Ng, mu_iN=muiN, Gamma_T=GT, nu_w=0.0)
    c = fl.coefficients(col, otab, T)
    Gf, Ef = fl.flux_and_field(col, c, n)
    cell = lambda f: 0.5 * (f + np.roll(f, 1))
    assert np.allclose(G, cell(Gf), rtol=1e-9, atol=1e-9 * np.abs(Gf).max())
    assert np.allclose(E, cell(Ef), rtol=1e-9, atol=1e-9 * np.abs(Ef).max())
    assert np.allclose(nu, c["nu_i"], rtol=1e-9)


def test_residuals_vanish_on_the_tabulated_closure():
    recs = uniform_records()
    tab = sc.Table(recs)
    n, T = state(seed=2)
    p = w.Params(gas_mass_amu=w.AMU_NE, pressure_torr=1.0, L_m=0.1, n_cells=256)
    Ng = cl.n_gas(p)
    muiN, GT = 1.3e22, 3e19
    G, H, nu, E = cl.table_closure(n, T, GT, p.L_m, Ng, muiN, tab)
    # a window in the fluid frame whose moments are the closure's, then put into the particle frame
    f = dict(n_e=n, mean_eps_e=1.5 * T, gamma_e=G, heat_e=H, iz_rate=nu * n, E=E,
             gamma_i=G + GT)                       # Gamma_i - Gamma_e = Gamma_T everywhere
    X, Y = cl.residual_samples(cl.mirror(f), p, tab, muiN)
    assert X.shape == (256, 15) and Y.shape == (256, 3)
    assert np.max(np.abs(Y[:, 0])) < 1e-5 * np.abs(G / n).max()
    assert np.max(np.abs(Y[:, 1])) < 1e-5 * np.abs(H / n).max()
    assert np.max(np.abs(Y[:, 2])) < 1e-5 * nu.max()
    assert np.allclose(X[:, 2], n / n.mean(), rtol=1e-6)
    assert np.allclose(X[:, 7], 1.5 * T, rtol=1e-6)
    assert np.allclose(X[:, 12], E / (Ng * 1e-21), rtol=1e-5)
    # stencil order: column d+2 holds cell j+d
    assert np.allclose(X[:, 3], np.roll(n / n.mean(), -1), rtol=1e-6)


def test_observables_of_a_travelling_growing_wave():
    # n = n0 (1 + a(t) cos(k x - w t)) with a = a0 exp(g t) capped at 0.3: lambda = L/m,
    # v_ph = w/k, gamma = g
    L, N, m, v, g = 0.1, 512, 7, 1500.0, 4e5
    k = 2 * np.pi * m / L
    x = np.arange(N) * L / N
    t = np.arange(1, 301) * 1e-7
    rng = np.random.default_rng(0)
    modes = []
    for ti in t:
        a = min(1e-4 * np.exp(g * ti), 0.3)
        n = 1e15 * (1 + a * np.cos(k * x - k * v * ti) + 1e-6 * rng.standard_normal(N))
        F = np.fft.fft(n) / N
        modes.append(np.concatenate([[n.mean()], F[1:33]]))
    o = sc.observables(t, np.array(modes), L)
    assert o["m"] == m
    assert o["lam"] == pytest.approx(L / m)
    assert o["v_ph"] == pytest.approx(v, rel=1e-6)
    assert o["gamma"] == pytest.approx(g, rel=1e-3)
