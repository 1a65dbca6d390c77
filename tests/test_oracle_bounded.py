"""Pins of the oracle's bounded column (Sec. V: cathode at x = 0 emitting the current
density J_e0, anode at x = L, both absorbing, the voltage across the gap): the
Dirichlet field against the paper's Thomas route and a closed form, particle
bookkeeping (absorbed, emitted), and the space-charge-limited current of a vacuum
diode, the Child-Langmuir law J = (4 eps0 / 9) (2e/m)^(1/2) V^(3/2) / d^2."""
import numpy as np
import pytest

import oracle
from paper_2202_03215_gb300 import workloads as w
from tests.helpers import QE, ME

EPS0 = 8.8541878128e-12


def test_dirichlet_field_matches_thomas_and_a_closed_form():
    rng = np.random.default_rng(4)
    N, dx, C = 200, 1e-4, 3.7e-9
    Qi = rng.integers(0, 2**40, N + 1)
    Qe = rng.integers(0, 2**40, N + 1)
    Eh = oracle.field_exact_bounded(Qi, Qe, C)
    # the paper's route: -phi_{j-1} + 2 phi_j - phi_{j+1} = dx^2 rho_j / eps0 on the interior nodes,
    # phi_0 = phi_N = 0 (the applied voltage enters separately), E_{j+1/2} = -(phi_{j+1} - phi_j) / dx
    rho = np.zeros(N)
    rho[1:] = (Qi[1:N] - Qe[1:N]).astype(float) * C * EPS0 / dx   # C = e w / (eps0 2^32) per unit Q
    phi = np.concatenate([oracle.poisson_thomas(rho, dx), [0.0]])
    Et = -(phi[1:] - phi[:-1]) / dx
    assert np.max(np.abs(Eh - Et)) < 1e-9 * np.max(np.abs(Et))
    assert abs(Eh.sum()) < 1e-9 * np.abs(Eh).sum()          # equal potential at both electrodes
    # uniform interior charge density rho0: E_{j+1/2} = rho0 (x_{j+1/2} - L/2) / eps0
    Qu = np.zeros(N + 1, np.int64)
    Qu[1:N] = 2**36
    Eu = oracle.field_exact_bounded(Qu, np.zeros(N + 1, np.int64), C)
    x = (np.arange(N) + 0.5) * dx
    rho0 = 2**36 * C * EPS0 / dx
    assert np.allclose(Eu, rho0 * (x - N * dx / 2) / EPS0, rtol=0, atol=1e-9 * np.abs(Eu).max())


def diode(J_emit, V, n_cells=100, L=0.01, dt=5e-12, T_emit=0.05, w_target=1e8, seed=3):
    # a vacuum gap: negligible gas (one elastic process at vanishing density), no ions
    n0 = 1000
    return w.Params(gas_mass_amu=w.AMU_AR, pressure_torr=1e-9, L_m=L, n_cells=n_cells, dt_s=dt,
                    drive=w.DRIVE_V, V_applied=V, n_e0=n0, n_i0=0, ion_subcycle=0, n0_m3=w_target * n0 / L,
                    Te0_eV=T_emit, loss_mode=w.LOSS_NONE, flags=w.FLAG_BOUNDED, J_emit_Am2=J_emit,
                    T_emit_eV=T_emit, capacity=200_000, seed=seed, eps_max_e_eV=500.0)


def test_bookkeeping_absorbed_and_emitted():
    p = diode(50.0, 100.0)
    o = oracle.Oracle(p)
    st0 = o.stats()
    o.step(400)
    st = o.stats()
    per_step = p.J_emit_Am2 * p.dt_s / (QE * p.n0_m3 * p.L_m / p.n_e0)
    assert st["emitted"] == int(np.floor(400 * per_step + 1e-9))
    assert st["n_e"] == p.n_e0 + st["emitted"] - sum(st["absorbed_e"])
    s = o.get_state()
    assert len(s["Q_e"]) == p.n_cells + 1
    assert s["Q_e"].sum() == st["n_e"] * 2**32          # every electron's charge on the N + 1 nodes
    assert np.all((s["cell_e"] >= 0) & (s["cell_e"] < p.n_cells))


def test_vacuum_diode_child_langmuir():
    V, d = 100.0, 0.01
    Jcl = 4 * EPS0 / 9 * np.sqrt(2 * QE / ME) * V ** 1.5 / d ** 2
    p = diode(4 * Jcl, V)
    o = oracle.Oracle(p)
    o.step(4000)                              # a few transit times (about 600 steps each)
    a0 = o.stats()["absorbed_e"][1]
    steps = 4000
    o.step(steps)
    wgt = p.n0_m3 * p.L_m / p.n_e0
    J = (o.stats()["absorbed_e"][1] - a0) * QE * wgt / (steps * p.dt_s)
    # space-charge limited: the anode receives the Child-Langmuir current (thermal emission
    # velocities at 0.05 eV raise it by a few per cent), the rest returns to the cathode
    assert J == pytest.approx(Jcl, rel=0.08)
    assert o.stats()["absorbed_e"][0] > 0


def test_emitted_electrons_are_a_half_maxwellian_at_the_cathode():
    """Cathode emission (Sec. V) at T_emit: the newborns of one step have v_x half-normal and
    v_y, v_z normal with sigma = (e T_emit / m)^(1/2), and start at x = u v_x dt with u uniform
    (the part of the step already flown)."""
    from scipy import stats
    T_emit = 2.0
    p = diode(1e4, 0.0, T_emit=T_emit)
    o = oracle.Oracle(p)
    id0 = o.get_state()["next_id"]
    o.step(1)
    s = o.get_state()
    new = s["id_e"] >= id0
    per_step = p.J_emit_Am2 * p.dt_s / (QE * p.n0_m3 * p.L_m / p.n_e0)
    assert new.sum() == int(np.floor(per_step)) > 2000
    sig = np.sqrt(QE * T_emit / ME)
    vx, vy, vz = s["vx_e"][new] / sig, s["vy_e"][new] / sig, s["vz_e"][new] / sig
    assert np.all(vx >= 0)
    assert stats.kstest(vx, "halfnorm").pvalue > 1e-4
    assert stats.kstest(np.concatenate([vy, vz]), "norm").pvalue > 1e-4
    dx = p.L_m / p.n_cells
    u = (s["cell_e"][new] + s["off_e"][new]) * dx / (s["vx_e"][new] * p.dt_s)
    assert stats.kstest(u, "uniform").pvalue > 1e-4
