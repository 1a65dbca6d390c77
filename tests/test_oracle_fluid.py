"""Pins of the oracle's fluid step (Sec. IV.A, eqs. 3-5, 8-9, 11, 17) against
closed forms: the homogeneous steady state, the von Neumann symbols of the
backward-Euler continuity and energy updates (textbook diffusion /
advection-diffusion-relaxation), and the exact particle and energy balances."""
import numpy as np
import pytest

from oracle import fluid as fl

N_GAS = 3.219e22


def const_table(muN=1e25, DN=5e25, mueN=1.6e25, DeN=8e25, nu_izN=2e-17, lossN=1e-14, dloss=0.0, nT=16):
    """Transport records whose resampled table is constant in Te except for
    a linear loss of slope dloss (per N, per eV) around Te = 4 eV."""
    recs = []
    for k in range(nT):
        Te = 2.0 + 4.0 * k / (nT - 1)
        recs.append(dict(mean_eps_eV=1.5 * Te, muN=muN, DN=DN, mueN=mueN, DeN=DeN, nu_izN=nu_izN,
                         lossN=lossN + dloss * (Te - 4.0)))
    return fl.make_table(recs, nT)


def column(L=0.3, Gamma_T=0.0, nu_w=None, tab=None, mu_iN=1.3e22):
    col = dict(L_m=L, N_gas=N_GAS, mu_iN=mu_iN, Gamma_T=Gamma_T, nu_w=0.0)
    col["nu_w"] = nu_w if nu_w is not None else float(fl.lookup(tab, np.array([4.0]))["nu_izN"][0] * N_GAS)
    return col


def test_homogeneous_steady_state_is_stationary():
    # nu_i(T0) = nu_w and P0 = n0 L(T0) with P0 = mu_e Gamma_T^2 / (n0 (mu_e + mu_i)^2)
    tab = const_table(dloss=4e-15)
    n0, T0 = 1e16, 4.0
    c = fl.coefficients(column(tab=tab), tab, np.array([T0]))
    mu_e, mu_i, L = c["mu_e"][0], c["mu_i"], c["L"][0]
    GT = n0 * (mu_e + mu_i) * np.sqrt(L / mu_e)
    col = column(Gamma_T=GT, tab=tab)
    n = np.full(256, n0)
    T = np.full(256, T0)
    for _ in range(50):
        n, T = fl.step(col, tab, n, T, 1e-8)
    assert np.max(np.abs(n / n0 - 1)) < 1e-12
    assert np.max(np.abs(T / T0 - 1)) < 1e-12


@pytest.mark.parametrize("m", [1, 7, 40])
def test_continuity_symbol(m):
    # uniform T: one step multiplies a density mode by
    # (1 + dt nu_i) / (1 + dt nu_w + 4 dt D_a sin^2(k dx/2) / dx^2), D_a = mu_i D_e/(mu_e + mu_i)
    tab = const_table()
    N, L, dt = 512, 0.3, 2e-8
    col = column(L=L, tab=tab, nu_w=1e4)
    dx = L / N
    mu_e, D_e, mu_i = 1e25 / N_GAS, 5e25 / N_GAS, 1.3e22 / N_GAS
    nu_i = 2e-17 * N_GAS
    Da = mu_i * D_e / (mu_e + mu_i)
    x = np.arange(N)
    n = 1e16 * (1 + 1e-3 * np.cos(2 * np.pi * m * x / N))
    n1, _ = fl.step(col, tab, n, np.full(N, 4.0), dt)
    g = (1 + dt * nu_i) / (1 + dt * 1e4 + 4 * dt * Da * np.sin(np.pi * m / N) ** 2 / dx ** 2)
    c0, c1 = fl.modes(n, m)[-1], fl.modes(n1, m)[-1]
    assert c1 / c0 == pytest.approx(g, rel=1e-9)
    if m != 1:     # no other mode is excited
        assert abs(fl.modes(n1, 1)[0]) < 1e-12 * n1.mean()
    assert n1.mean() == pytest.approx(1e16 * (1 + dt * nu_i) / (1 + dt * 1e4), rel=1e-12)


@pytest.mark.parametrize("m,GT,dloss", [(3, 0.0, 0.0), (3, 2e20, 0.0), (25, 2e20, 6e-15)])
def test_energy_symbol(m, GT, dloss):
    # uniform n, E = Gamma_T/(n (mu_e + mu_i)) uniform: one step multiplies a temperature mode by
    # 1 / (1 - i dt mu_eps E sin(k dx)/dx + 4 dt D_eps sin^2(k dx/2)/dx^2 + (2/3) dt L')
    tab = const_table(lossN=0.0, dloss=dloss)       # L(4 eV) = 0: the mean temperature stays in the table
    N, L, dt, n0 = 256, 0.3, 1e-8, 1e16
    col = column(L=L, Gamma_T=GT, tab=tab)
    dx = L / N
    mu_e, mu_i = 1e25 / N_GAS, 1.3e22 / N_GAS
    mu_eps, D_eps = 1.6e25 / N_GAS, 8e25 / N_GAS
    E0 = GT / (n0 * (mu_e + mu_i))
    x = np.arange(N)
    T = 4.0 + 1e-3 * np.cos(2 * np.pi * m * x / N)
    _, T1 = fl.step(col, tab, np.full(N, n0), T, dt)
    th = 2 * np.pi * m / N
    g = 1.0 / (1 - 1j * dt * mu_eps * E0 * np.sin(th) / dx + 4 * dt * D_eps * np.sin(th / 2) ** 2 / dx ** 2
               + 2.0 / 3.0 * dt * dloss * N_GAS)
    c0, c1 = fl.modes(T, m)[-1], fl.modes(T1, m)[-1]
    assert abs(c1 / c0 - g) < 1e-9 * abs(g)


def neon_table():
    from paper_2202_03215_gb300 import workloads as w
    from oracle import two_term as tt
    xo = [(x.kind, x.threshold_eV, x.energy_eV, x.sigma_m2) for x in w.neon_xsecs() if x.kind <= 2]
    recs = []
    for en in np.geomspace(3, 150, 24):
        r = tt.solve(xo, w.AMU_NE, en, eps_max=150.0, n=600)
        recs.append(dict(mean_eps_eV=r["mean_eps"], muN=r["muN"], DN=r["DN"], mueN=r["mueN"], DeN=r["DeN"],
                         nu_izN=r["nu_izN"], lossN=r["loss_N"]))
    return fl.make_table(recs, 64)


def test_particle_and_energy_balance():
    # fluxes telescope: sum n' (1 + dt nu_w) - sum n = dt sum n nu_i; the energy changes by
    # dt sum (P - n' (L + L'(T' - T))) exactly (periodic column)
    tab = neon_table()
    rng = np.random.default_rng(5)
    N, dt = 512, 2e-8
    col = column(L=0.1, Gamma_T=2e20, tab=tab, nu_w=3e4)
    n = 1e16 * (1 + 0.05 * rng.standard_normal(N))
    T = 5.0 + 0.3 * rng.standard_normal(N)
    c = fl.coefficients(col, tab, T)
    n1, T1 = fl.step(col, tab, n, T, dt)
    assert n1.sum() * (1 + dt * col["nu_w"]) - n.sum() == pytest.approx(dt * np.sum(n * c["nu_i"]), rel=1e-9)
    Gam, E = fl.flux_and_field(col, c, n1)
    P = -0.5 * (Gam * E + np.roll(Gam * E, 1))
    if np.all((T1 > tab["T0"]) & (T1 < tab["T0"] + (tab["nT"] - 1) * tab["dT"])):
        lhs = 1.5 * (np.sum(n1 * T1) - np.sum(n * T))
        rhs = dt * np.sum(P - n1 * (c["L"] + c["dL"] * (T1 - T)))
        assert lhs == pytest.approx(rhs, rel=1e-8)


def test_pair_losses_conserve_the_particle_number():
    # with pair losses the column loses exactly what it ionizes: sum n' = sum n
    tab = neon_table()
    rng = np.random.default_rng(6)
    N, dt = 256, 2e-8
    col = column(L=0.1, Gamma_T=2e20, tab=tab, nu_w=0.0)
    col["pair"] = True
    n = 1e16 * (1 + 0.1 * rng.standard_normal(N))
    T = 5.5 + 0.5 * rng.standard_normal(N)
    corr = np.stack([np.zeros(N), np.zeros(N), 1e5 * rng.standard_normal(N)])
    for c in (None, corr):
        n1, _ = fl.step(col, tab, n, T, dt, corr=c)
        assert n1.sum() == pytest.approx(n.sum(), rel=1e-12)


def test_cyclic_solve_against_dense():
    rng = np.random.default_rng(1)
    N = 33
    lo, up = -rng.random(N), -rng.random(N)
    dg = 2.5 + rng.random(N)
    rhs = rng.standard_normal(N)
    A = np.diag(dg)
    for j in range(N):
        A[j, (j - 1) % N] += lo[j]
        A[j, (j + 1) % N] += up[j]
    assert np.allclose(fl.cyclic_solve(lo, dg, up, rhs), np.linalg.solve(A, rhs), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("pair", [False, True])
def test_the_model_is_linear_in_the_density(pair):
    """The fluid model, like the particle model (Sec. II), is linear in the plasma density: four
    times the density and the current (an exact power of two) give four times the density and
    the same temperature, bit for bit, through both tridiagonal solves and the field."""
    tab = const_table(dloss=4e-15)
    rng = np.random.default_rng(12)
    n = 1e16 * (1 + 0.05 * rng.standard_normal(512))
    T = 4.0 + 0.2 * rng.standard_normal(512)
    c = fl.coefficients(column(tab=tab), tab, np.array([4.0]))   # the current of the steady state at 4 eV
    GT = 1e16 * (c["mu_e"][0] + c["mu_i"]) * np.sqrt(c["L"][0] / c["mu_e"][0])
    c1 = column(Gamma_T=GT, tab=tab)
    c4 = dict(c1, Gamma_T=4 * c1["Gamma_T"])
    if pair:
        c1["pair"] = c4["pair"] = True
    n1, T1, n4, T4 = n.copy(), T.copy(), 4 * n, T.copy()
    lo, hi = tab["T0"], tab["T0"] + (tab["nT"] - 1) * tab["dT"]
    for _ in range(30):
        n1, T1 = fl.step(c1, tab, n1, T1, 2e-8)
        n4, T4 = fl.step(c4, tab, n4, T4, 2e-8)
        assert np.array_equal(n4, 4 * n1) and np.array_equal(T4, T1)
        assert np.all((T1 > lo) & (T1 < hi))          # no clipping at the table ends masks a difference
    assert np.std(n1) > 0 and not np.array_equal(n1, n)


@pytest.mark.parametrize("m,v", [(2, 3e3), (17, -8e3), (60, 2e4)])
def test_flux_correction_is_implicit_upwind_advection(m, v):
    # no diffusion, drift, ionization or losses: the continuity step with a flux correction of
    # g = v per electron is backward-Euler first-order upwind advection, which multiplies the mode
    # exp(i theta j) by 1 / (1 + (dt |v| / dx)(1 - exp(-+ i theta))) (- for v > 0: the upwind
    # cell is j - 1), conserving the particle number
    tab = const_table(DN=0.0, nu_izN=0.0, lossN=0.0)
    N, L, dt = 256, 0.1, 2e-8
    col = column(L=L, tab=tab, nu_w=0.0)
    dx = L / N
    x = np.arange(N)
    n = 1e16 * (1 + 1e-2 * np.cos(2 * np.pi * m * x / N))
    corr = np.stack([np.full(N, v), np.zeros(N), np.zeros(N)])
    n1, _ = fl.step(col, tab, n, np.full(N, 4.0), dt, corr=corr)
    th = 2 * np.pi * m / N
    g = 1.0 / (1.0 + dt * abs(v) / dx * (1 - np.exp(-np.sign(v) * 1j * th)))
    c0, c1 = fl.modes(n, m)[-1], fl.modes(n1, m)[-1]
    assert abs(c1 / c0 - g) < 1e-9 * abs(g)
    assert n1.sum() == pytest.approx(n.sum(), rel=1e-13)


def test_flux_correction_keeps_the_density_positive():
    # a correction velocity that changes sign from cell to cell (converging and diverging faces)
    # at a Courant number of 5: the upwind matrix is an M-matrix, n' > 0, the number conserved
    tab = const_table(DN=0.0, nu_izN=0.0, lossN=0.0)
    N, L, dt = 128, 0.1, 2e-8
    col = column(L=L, tab=tab, nu_w=0.0)
    rng = np.random.default_rng(8)
    v = 5 * (L / N) / dt * rng.standard_normal(N)
    n = 1e16 * (1 + 0.5 * rng.random(N))
    n1, _ = fl.step(col, tab, n, np.full(N, 4.0), dt, corr=np.stack([v, np.zeros(N), np.zeros(N)]))
    assert np.all(n1 > 0)
    assert n1.sum() == pytest.approx(n.sum(), rel=1e-12)


@pytest.mark.parametrize("m,w", [(3, 5e3), (31, -2e4)])
def test_energy_flux_correction_is_implicit_upwind_advection(m, w):
    # uniform n, no field, conduction, energy drift or loss: an energy-flux correction of
    # h = w T per electron is backward-Euler upwind advection of (3/2) n T with velocity w,
    # which multiplies a temperature mode by 1 / (1 + (2/3)(dt |w| / dx)(1 - exp(-+ i theta)))
    tab = const_table(mueN=0.0, DeN=0.0, lossN=0.0, nu_izN=0.0)
    N, L, dt, n0 = 256, 0.1, 1e-8, 1e16
    col = column(L=L, tab=tab, nu_w=0.0)
    dx = L / N
    x = np.arange(N)
    T = 4.0 + 1e-2 * np.cos(2 * np.pi * m * x / N)
    corr = np.stack([np.zeros(N), w * T, np.zeros(N)])
    n1, T1 = fl.step(col, tab, np.full(N, n0), T, dt, corr=corr)
    assert np.allclose(n1, n0, rtol=1e-13)
    th = 2 * np.pi * m / N
    g = 1.0 / (1.0 + 2.0 / 3.0 * dt * abs(w) / dx * (1 - np.exp(-np.sign(w) * 1j * th)))
    c0, c1 = fl.modes(T, m)[-1], fl.modes(T1, m)[-1]
    assert abs(c1 / c0 - g) < 1e-9 * abs(g)
    assert T1.mean() == pytest.approx(T.mean(), rel=1e-12)
