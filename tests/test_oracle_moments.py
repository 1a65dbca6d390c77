"""Pins of the oracle's diagnostic moments (Fig. 4 quantities: densities, fluxes, mean energy,
heat flux, ionization rate, field and potential) by properties that their definitions fix,
independent of how the oracle accumulates them:

- cloud-in-cell weights sum to one, so the integral over the column of n, Gamma = n <v_x> and
  H = n <eps v_x> equals the macro-weight times the count, sum v_x and sum eps v_x of the particles
  the step leaves;
- the potential obeys Poisson's equation (Sec. II) against the sampled charge density, and the
  node field is minus its centred difference minus the applied field E0;
- a mono-energetic swarm has that mean energy at every node it occupies;
- the ionization rate integrates to the births per unit area and time."""
import numpy as np
import pytest

import oracle
from paper_2202_03215_gb300 import workloads as w
from tests.helpers import QE, ME, AMU, EPS0, beam_state


def _collisionless(n, N=64, L=0.02, E0=300.0, **kw):
    base = dict(gas_mass_amu=w.AMU_AR, L_m=L, n_cells=N, dt_s=2e-11, xsec=[], field_mode=w.FIELD_POISSON,
                drive=w.DRIVE_E0, E0_Vpm=E0, n_e0=n, n_i0=n, ion_subcycle=1, loss_mode=w.LOSS_NONE,
                diag_every=1, n0_m3=1e15, Te0_eV=3.0, Ti0_eV=0.5, seed=21)
    base.update(kw)
    return w.Params(**base)


def _sums(o, M_i):
    s = o.get_state()
    out = {}
    for sp, m in (("e", ME), ("i", M_i)):
        v2 = s[f"vx_{sp}"] ** 2 + s[f"vy_{sp}"] ** 2 + s[f"vz_{sp}"] ** 2
        eps = 0.5 * m / QE * v2
        out[sp] = (len(s[f"vx_{sp}"]), s[f"vx_{sp}"].sum(), (eps * s[f"vx_{sp}"]).sum())
    return out


@pytest.mark.parametrize("f32", [False, True])
def test_column_integrals_of_densities_and_fluxes(f32):
    p = _collisionless(6000, precision=w.MIXED if f32 else w.FP64)
    o = oracle.Oracle(p, f32=f32)
    d = o.derived()
    wgt, dx = d["w"], d["dx"]
    acc = {"e": np.zeros(3), "i": np.zeros(3)}
    K = 5
    for _ in range(K):
        o.step(1)
        for sp, t in _sums(o, w.AMU_AR * AMU).items():
            acc[sp] += t
    m = o.moments()
    assert m["n_samples"] == K
    for sp, n_key, g_key in (("e", "n_e", "gamma_e"), ("i", "n_i", "gamma_i")):
        cnt, sv, sev = acc[sp] / K
        assert m[n_key].sum() * dx == pytest.approx(cnt * wgt, rel=1e-12)
        scale = np.abs(m[g_key]).sum() * dx
        assert abs(m[g_key].sum() * dx - sv * wgt) <= 1e-9 * scale
        if sp == "e":
            hs = np.abs(m["heat_e"]).sum() * dx
            assert abs(m["heat_e"].sum() * dx - sev * wgt) <= 1e-6 * hs   # eps in the storage precision
    assert np.abs(m["gamma_e"]).max() > 0 and np.abs(m["gamma_i"]).max() > 0


@pytest.mark.parametrize("loss", [w.LOSS_NONE, w.LOSS_RADIAL])
def test_potential_obeys_poisson_against_the_sampled_density(loss):
    # RADIAL makes the column non-neutral: the uniform background (the mean charge) is removed
    p = _collisionless(5000, loss_mode=loss, nu_w=5e8 if loss == w.LOSS_RADIAL else 0.0)
    o = oracle.Oracle(p)
    o.step(7)
    m = o.moments()
    dx = o.derived()["dx"]
    phi, E = m["phi"], m["E"]
    rho = QE * (m["n_i"] - m["n_e"])
    rho = rho - rho.mean()
    lap = (np.roll(phi, -1) - 2 * phi + np.roll(phi, 1)) / dx**2
    assert np.abs(rho).max() > 0
    assert np.max(np.abs(lap + rho / EPS0)) <= 1e-8 * np.abs(rho / EPS0).max()
    assert phi[0] == 0.0
    grad = -(np.roll(phi, -1) - np.roll(phi, 1)) / (2 * dx)
    assert np.max(np.abs(E + p.E0_Vpm - grad)) <= 1e-8 * np.abs(grad).max()


def test_monoenergetic_swarm_mean_energy():
    n, N, eps0 = 4000, 64, 7.5
    p = _collisionless(n, N=N, field_mode=w.FIELD_APPLIED, E0_Vpm=0.0, n_i0=0, ion_subcycle=0)
    o = oracle.Oracle(p)
    rng = np.random.default_rng(3)
    st = beam_state(n, N, np.sqrt(2 * QE * eps0 / ME), rng, direction=(1.0, -2.0, 0.5))
    o.set_state(st)
    o.step(3)
    m = o.moments()
    occ = m["n_e"] > 0
    assert occ.sum() == N
    assert np.allclose(m["mean_eps_e"][occ], eps0, rtol=1e-12, atol=0)


def test_ionization_rate_integrates_to_the_births():
    p = w.config_argon_small(seed=4, n_e0=20000, n_i0=20000, diag_every=5, E0_Vpm=2500.0, drive=w.DRIVE_E0)
    o = oracle.Oracle(p)
    o.step(40)
    st, m, d = o.stats(), o.moments(), o.derived()
    assert st["births"] > 0
    assert m["n_steps"] == 40
    rate = st["births"] * d["w"] / (40 * p.dt_s)   # ionization events per m^2 per s
    assert m["iz_rate"].sum() * d["dx"] == pytest.approx(rate, rel=1e-12)
