"""T4/T7 pins of the oracle's null-collision Monte Carlo collisions: real
collision counts per process against the analytic collision frequencies,
the constant-frequency (Maxwell) model, and the scattering kinematics."""
import numpy as np
import pytest
from scipy import stats

import oracle
from paper_2202_03215_gb300 import workloads as w
from tests.helpers import QE, ME, AMU, KB, beam_state, maxwell_model_xsec, n_gas


def _sigma(x, eps):
    s = np.interp(eps, x.energy_eV, x.sigma_m2)
    if x.kind in (w.EXCITATION, w.IONIZATION) and eps < x.threshold_eV:
        return 0.0
    return float(s)


def _beam_params(n, **kw):
    base = dict(L_m=0.05, n_cells=500, dt_s=2e-11, field_mode=w.FIELD_APPLIED, drive=w.DRIVE_E0,
                E0_Vpm=0.0, n_e0=n, n_i0=0, ion_subcycle=0, loss_mode=w.LOSS_NONE, Te0_eV=1.0,
                capacity=2 * n + 10)
    base.update(kw)
    return w.Params(**base)


@pytest.mark.parametrize("eps0", [10.0, 30.0, 120.0])
def test_real_collision_counts_match_analytic_rates(eps0):
    n = 200_000
    p = _beam_params(n)
    o = oracle.Oracle(p)
    speed = np.sqrt(2 * QE * eps0 / ME)
    o.set_state(beam_state(n, p.n_cells, speed, np.random.default_rng(1)))
    o.step(1)
    codes = o.codes(0, n)
    ng = n_gas()
    # energy-binned majorant: the larger summed frequency at the two ends of the table bin holding eps0
    de = p.eps_max_e_eV / (p.n_table - 1)
    i = int(eps0 / de)
    ends = [(i * de), ((i + 1) * de)]
    S = [sum(_sigma(x, e) for x in p.xsec[:3]) * ng * np.sqrt(2 * QE * e / ME) for e in ends]
    nub = max(S)
    Pn = 1 - np.exp(-nub * p.dt_s)
    for k, x in enumerate(p.xsec[:3]):
        nu = ng * _sigma(x, eps0) * speed
        pk = Pn * nu / nub
        cnt = np.count_nonzero(codes == k)
        if pk == 0:
            assert cnt == 0
        else:
            assert abs(cnt - n * pk) < 4.5 * np.sqrt(n * pk * (1 - pk)), (k, cnt, n * pk)
    # the candidates are the particles of the bin with probability P_null(bin): real + null
    d = o.derived()
    nus = d["nu_star_e"]
    # nu* bounds the total frequency on the whole table range
    e = np.linspace(0, p.eps_max_e_eV, 20001)
    tot = sum(np.array([_sigma(x, ee) for ee in e]) for x in p.xsec[:3]) * ng * np.sqrt(2 * QE * e / ME)
    assert nus >= tot.max() * (1 - 1e-4)


def test_maxwell_model_has_no_energy_dependence():
    n, nu = 200_000, 4e9
    xs = [maxwell_model_xsec(nu, n_gas(), 100.0, 8193)]
    p = _beam_params(n, xsec=xs, eps_max_e_eV=100.0, Te0_eV=3.0)
    o = oracle.Oracle(p)
    o.step(1)
    codes = o.codes(0, n)
    P = 1 - np.exp(-nu * p.dt_s)
    cnt = np.count_nonzero(codes == 0)
    assert abs(cnt - n * P) < 4.5 * np.sqrt(n * P * (1 - P))
    assert abs(o.derived()["nu_star_e"] / nu - 1) < 1e-9


def test_elastic_kinematics_isotropic_with_mass_ratio_loss():
    n, eps0 = 200_000, 10.0
    M_amu = 0.01   # light gas so that 2m/M is resolved
    p = _beam_params(n, gas_mass_amu=M_amu)
    o = oracle.Oracle(p)
    speed = np.sqrt(2 * QE * eps0 / ME)
    o.set_state(beam_state(n, p.n_cells, speed, np.random.default_rng(2)))
    o.step(1)
    codes = o.codes(0, n)
    s = o.get_state()
    sel = codes == 0
    v = np.stack([s["vx_e"][sel], s["vy_e"][sel], s["vz_e"][sel]])
    eps = 0.5 * ME / QE * (v * v).sum(0)
    em = 2 * ME / (M_amu * AMU)
    r = eps / eps0                       # = 1 - em (1 - cos chi), cos chi ~ U(-1, 1)
    assert stats.kstest((r - (1 - 2 * em)) / (2 * em), "uniform").pvalue > 1e-4
    nvec = v / np.sqrt((v * v).sum(0))
    m = nvec.shape[1]
    assert np.all(np.abs(nvec.mean(1)) < 5 / np.sqrt(3 * m))
    assert np.all(np.abs((nvec ** 2).mean(1) - 1 / 3) < 5 * np.sqrt(4 / 45 / m))
    # cos chi against the beam direction (+x) is uniform
    assert stats.kstest((nvec[0] + 1) / 2, "uniform").pvalue > 1e-4


def test_excitation_and_ionization_energy_balance():
    n, eps0 = 200_000, 60.0
    p = _beam_params(n)
    o = oracle.Oracle(p)
    speed = np.sqrt(2 * QE * eps0 / ME)
    o.set_state(beam_state(n, p.n_cells, speed, np.random.default_rng(3)))
    o.step(1)
    codes = o.codes(0, n)
    s = o.get_state()
    K = 0.5 * ME / QE
    eps = K * (s["vx_e"] ** 2 + s["vy_e"] ** 2 + s["vz_e"] ** 2)
    exc = codes == 1
    assert np.allclose(eps[:n][exc], eps0 - 11.5, rtol=1e-12)
    iz = np.nonzero(codes == 2)[0]
    nb = len(iz)
    assert s["n_e"] == n + nb and s["n_i"] == nb
    ej = eps[n:n + nb]                   # newborns appended in parent-slot order
    assert np.allclose(eps[iz] + ej, eps0 - 15.76, rtol=1e-11)
    assert stats.kstest(ej / (eps0 - 15.76), "uniform").pvalue > 1e-4
    # newborn electron sits at its parent's position, the ion too
    assert np.array_equal(s["cell_e"][n:], s["cell_e"][iz]) and np.array_equal(s["off_e"][n:], s["off_e"][iz])
    assert np.array_equal(s["cell_i"], s["cell_e"][iz])
    # newborn ion velocity: gas Maxwellian
    M = p.gas_mass_amu * AMU
    vt = np.sqrt(KB * p.T_gas_K / M)
    vi = np.concatenate([s["vx_i"], s["vy_i"], s["vz_i"]]) / vt
    assert stats.kstest(vi, "norm").pvalue > 1e-4


def test_ion_charge_exchange_takes_the_neutral_velocity():
    n = 100_000
    p = _beam_params(0, n_i0=n, ion_subcycle=1, capacity=n + 10, xsec=w.argon_xsecs(sigma_iso=0.0))
    o = oracle.Oracle(p)
    M = p.gas_mass_amu * AMU
    g = 3000.0
    st = beam_state(0, p.n_cells, 0.0, np.random.default_rng(4), n_i=n, ion_speed=g)
    o.set_state(st)
    o.step(1)
    codes = o.codes(1, n)
    s = o.get_state()
    cx = codes == 3
    ng = n_gas()
    d = o.derived()
    # the relative speed varies with the neutral draw: compare with the mean of sigma g over the gas
    vt = np.sqrt(KB * p.T_gas_K / M)
    rng = np.random.default_rng(9)
    vn = rng.standard_normal((3, 400000)) * vt
    gr = np.sqrt((g - vn[0]) ** 2 + vn[1] ** 2 + vn[2] ** 2)
    nu_mean = ng * 5e-19 * gr.mean()
    P = (1 - np.exp(-d["nu_star_i"] * p.dt_s)) * nu_mean / d["nu_star_i"]
    assert abs(cx.sum() - n * P) < 4.5 * np.sqrt(n * P)
    vi = np.concatenate([s["vx_i"][cx], s["vy_i"][cx], s["vz_i"][cx]]) / vt
    assert stats.kstest(vi, "norm").pvalue > 1e-4


def test_ion_isotropic_scattering_in_the_centre_of_mass_frame():
    """Isotropic elastic ion-atom scattering (Sec. II) between equal masses: in a nearly cold gas
    (T_g = 3e-4 K, the gas density of 1 Torr at 300 K) a beam ion of speed g0 leaves with
    v' = v/2 + (g0/2) n, n uniform on the sphere, so |v' - v/2| = g0/2, the x-component of n is
    uniform on [-1, 1] (Archimedes) and its azimuth uniform; the count of scatterings is binomial
    with P_null nu_iso(g0)/nu*."""
    n, g0, s_iso = 200_000, 3000.0, 2e-19
    ge = np.array([0.0, 50.0])
    p = _beam_params(0, n_i0=n, ion_subcycle=1, capacity=n + 10, dt_s=5e-9, T_gas_K=3e-4,
                     pressure_torr=1e-6, xsec=[w.XSec(w.ION_ISO, ge, np.array([s_iso, s_iso]))])
    o = oracle.Oracle(p)
    st = beam_state(0, p.n_cells, 0.0, np.random.default_rng(6), n_i=n, ion_speed=g0)
    o.set_state(st)
    o.step(1)
    codes = o.codes(1, n)
    s = o.get_state()
    hit = codes == 0
    d = o.derived()
    assert d["n_g"] == pytest.approx(n_gas(1.0, 300.0), rel=1e-12)
    M = p.gas_mass_amu * AMU
    nu_iso = d["n_g"] * s_iso * g0
    P = d["P_null_i"] * nu_iso / d["nu_star_i"]
    assert abs(hit.sum() - n * P) < 4.5 * np.sqrt(n * P)
    assert hit.sum() > 5000
    # ions that did not scatter keep their velocity
    assert np.all(s["vx_i"][~hit] == g0) and not s["vy_i"][~hit].any()
    ux, uy, uz = s["vx_i"][hit] - g0 / 2, s["vy_i"][hit], s["vz_i"][hit]
    vt = np.sqrt(KB * p.T_gas_K / M)   # the neutrals' thermal speed, 0.25 m/s
    assert np.allclose(np.sqrt(ux**2 + uy**2 + uz**2), g0 / 2, rtol=0, atol=10 * vt)
    assert stats.kstest(ux / (g0 / 2), "uniform", args=(-1.0, 2.0)).pvalue > 1e-4
    assert stats.kstest(np.arctan2(uz, uy), "uniform", args=(-np.pi, 2 * np.pi)).pvalue > 1e-4


def test_energies_above_the_table_hold_its_last_value_and_are_counted():
    """Electrons above the table's range (eps_max_e) collide with the frequencies of the table's
    end and the last bin's majorant, and every collision candidate among them is counted as an
    overflow; below the range nothing is counted."""
    n, eps0 = 200_000, 600.0
    p = _beam_params(n, eps_max_e_eV=500.0)
    o = oracle.Oracle(p)
    o.set_state(beam_state(n, p.n_cells, np.sqrt(2 * QE * eps0 / ME), np.random.default_rng(8)))
    o.step(1)
    codes, st = o.codes(0, n), o.stats()
    ng = n_gas()
    de = p.eps_max_e_eV / (p.n_table - 1)
    ends = [(p.n_table - 2) * de, (p.n_table - 1) * de]
    S = [sum(_sigma(x, e) for x in p.xsec[:3]) * ng * np.sqrt(2 * QE * e / ME) for e in ends]
    Pn = 1 - np.exp(-max(S) * p.dt_s)
    cand = st["overflow_e"]
    assert abs(cand - n * Pn) < 4.5 * np.sqrt(n * Pn * (1 - Pn))
    v_end = np.sqrt(2 * QE * p.eps_max_e_eV / ME)     # the frequency held is the one at eps_max
    for k, x in enumerate(p.xsec[:3]):
        pk = Pn * ng * _sigma(x, p.eps_max_e_eV) * v_end / max(S)
        cnt = np.count_nonzero(codes == k)
        assert abs(cnt - n * pk) < 4.5 * np.sqrt(n * pk * (1 - pk)) + 1, (k, cnt, n * pk)
    # the same beam inside the range: no overflow
    o2 = oracle.Oracle(_beam_params(n, eps_max_e_eV=700.0))
    o2.set_state(beam_state(n, p.n_cells, np.sqrt(2 * QE * eps0 / ME), np.random.default_rng(8)))
    o2.step(1)
    assert o2.stats()["overflow_e"] == 0


def test_ions_above_the_table_are_counted():
    """Ions whose relative energy 0.5 M g^2/e exceeds eps_max_i (a nearly cold gas, 60 eV against a
    50 eV table): every candidate, drawn with the global P_null of the ions, is an overflow, and
    charge exchange keeps the table's end frequency."""
    n, eps_g = 200_000, 60.0
    p = _beam_params(0, n_i0=n, ion_subcycle=1, capacity=n + 10, T_gas_K=3e-4, pressure_torr=1e-6,
                     eps_max_i_eV=50.0, xsec=w.argon_xsecs(sigma_iso=0.0))
    o = oracle.Oracle(p)
    g = np.sqrt(2 * QE * eps_g / (p.gas_mass_amu * AMU))
    o.set_state(beam_state(0, p.n_cells, 0.0, np.random.default_rng(10), n_i=n, ion_speed=g))
    o.step(1)
    d, st, codes = o.derived(), o.stats(), o.codes(1, n)
    P = d["P_null_i"]
    assert abs(st["overflow_i"] - n * P) < 4.5 * np.sqrt(n * P * (1 - P))
    # CX (5e-19 m^2, constant) at the end of the table: nu = n_g sigma g_max with 0.5 M g_max^2 = e eps_max_i
    g_end = np.sqrt(2 * QE * p.eps_max_i_eV / (p.gas_mass_amu * AMU))
    pcx = P * d["n_g"] * 5e-19 * g_end / d["nu_star_i"]
    cnt = np.count_nonzero(codes == 3)
    assert abs(cnt - n * pcx) < 4.5 * np.sqrt(n * pcx * (1 - pcx))


@pytest.mark.parametrize("gas", ["argon", "neon_multilevel"])
def test_collision_frequency_tables_on_the_uniform_grid(gas):
    """The tables hold nu_k(eps_i) = n_g sigma_k(eps_i) v(eps_i) at eps_i = i eps_max/(n-1), with
    sigma linear between the given points, end values held, zero below an inelastic threshold;
    v = (2 e eps/m) for electrons and the relative speed (2 e eps/M) for ions."""
    xs = w.argon_xsecs(sigma_iso=1e-19) if gas == "argon" else w.neon_multilevel_xsecs()
    mass = w.AMU_AR if gas == "argon" else w.AMU_NE
    p = _beam_params(10, gas_mass_amu=mass, xsec=xs, n_table=4097)
    o = oracle.Oracle(p)
    ng = o.derived()["n_g"]
    assert ng == pytest.approx(n_gas(), rel=1e-12)
    e_proc = [x for x in xs if x.kind in (w.ELASTIC, w.EXCITATION, w.IONIZATION)]
    i_proc = [x for x in xs if x.kind in (w.ION_CX, w.ION_ISO)]
    for sp, procs, emax, m in ((0, e_proc, p.eps_max_e_eV, ME), (1, i_proc, p.eps_max_i_eV, mass * AMU)):
        eps = np.arange(p.n_table) * (emax / (p.n_table - 1))
        v = np.sqrt(2 * QE * eps / m)
        for j, x in enumerate(procs):
            s = np.interp(eps, x.energy_eV, x.sigma_m2)
            if x.kind in (w.EXCITATION, w.IONIZATION):
                s = np.where(eps < x.threshold_eV, 0.0, s)
            got = o.nu_table(sp, j)
            assert np.allclose(got, ng * s * v, rtol=1e-12, atol=0), (sp, j)
            if x.kind in (w.EXCITATION, w.IONIZATION):
                assert not got[eps < x.threshold_eV].any() and got[eps > x.threshold_eV + 1].all()


def test_real_collision_probability_is_the_continuous_time_one():
    """Null-collision method (Sec. II): with a majorant nu_b >= nu the per-step probability of a real
    collision, P(nu_b dt) nu/nu_b with P(x) = 1 - exp(-x), differs from the exact probability
    1 - exp(-nu dt) of the continuous-time process by at most (nu_b dt)^2/8 (from (1 - e^-x)/x,
    decreasing with slope above -1/2), and never exceeds it.  Measured from mono-energetic beams
    across the whole table, each energy's nu = n_g sum_k sigma_k(eps) v(eps) taken from the cross
    sections as given, not from the oracle's tables; nu_b is bounded by the global maximum nu*, so
    the bound does not assume the binned construction.  A candidate probability taken as nu_b dt,
    or a majorant below the frequency somewhere in a bin, fails it."""
    n = 400_000
    p = _beam_params(n, dt_s=2e-11)
    ng = n_gas()
    d0 = oracle.Oracle(p.with_(n_e0=10, capacity=20)).derived()
    x_star = d0["nu_star_e"] * p.dt_s
    assert 0.2 < x_star <= 0.3           # large enough to make the O(x^2) term visible
    rng = np.random.default_rng(31)
    worst = 0.0
    for eps0 in np.geomspace(0.05, 480.0, 23):
        o = oracle.Oracle(p)
        speed = np.sqrt(2 * QE * eps0 / ME)
        o.set_state(beam_state(n, p.n_cells, speed, rng))
        o.step(1)
        real = np.count_nonzero(o.codes(0, n) >= 0)
        nu = sum(_sigma(x, eps0) for x in p.xsec[:3]) * ng * speed
        exact = -np.expm1(-nu * p.dt_s)
        got = real / n
        sd = np.sqrt(max(exact, 1.0 / n) * (1 - exact) / n)
        # the table interpolates n_g sigma v linearly between grid points 0.06 eV apart
        slack = 2e-3 * exact
        assert got <= exact + 4.5 * sd + slack, (eps0, got, exact)
        assert exact - got <= x_star ** 2 / 8 + 4.5 * sd + slack, (eps0, got, exact, x_star)
        worst = max(worst, (exact - got) / (x_star ** 2 / 8))
    assert worst < 1.0
