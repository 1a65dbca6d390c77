"""Screen of discharge conditions with the fluid model, and the striation
observables used to judge it against the particle model (Sec. IV).

  * transport(): the closure tables -- two-term transport records at reduced
    fields on a log grid (pic_two_term, eqs. 6-9);
  * homogeneous_E0() / homogeneous_R(): the uniform steady state of eqs. 3-4
    (Sec. IV.A: nu_i(T0) = nu_w, P0 = n0 L_eps(T0)), either for an imposed
    field E0 with the wall loss equal to the ionization frequency (the
    particle model's pair-loss column) or for a tube of radius R with
    nu_w = D_a (2.405/R)^2 (eq. 2) and a current I;
  * linear(): growth rate, wave number and phase velocity of the fastest
    mode from the linearised fluid model, eqs. (19)-(22), and the instability
    criterion eq. (23);
  * observables(): wavelength, phase velocity and growth rate from a record
    of spatial Fourier modes of n_e(x, t): lambda = L/m* with m* the mode of
    largest time-averaged power over the saturated half of the record,
    v_ph = -(d phase/dt)/k from the unwrapped phase of m*, gamma = slope of
    ln|n_m*| while its amplitude lies between 10x its initial level and
    1/10 of its saturated level;
  * fluid_screen(): many columns of the fluid model in one batch on the GPU.

Every density is handled per unit density: the fluid model is linear in n
(Sec. II), so the current only scales n0.
"""
from __future__ import annotations

import json
import math
from dataclasses import dataclass
from typing import List, Sequence

import numpy as np

from . import Fluid, two_term
from . import workloads as w

KB = 1.380649e-23
QE = 1.602176634e-19
TORR = 133.32236842105263
# Reduced ion mobility of the particle model's neon ions (constant charge-exchange cross
# section 3e-19 m^2): mu_i N = A / sqrt(1 + (E/N)/x0) fitted to the ion drift of uniform
# particle-model columns at 19-62 Td (1.39e22 at 18.6 Td ... 0.79e22 at 62 Td, within 10 %);
# the form has the E^(-1/2) high-field law of a constant mean free path
MU_I_FIT_NEON = (4.37e22, 2.1)


def mu_iN_neon(EN_Td: float) -> float:
    A, x0 = MU_I_FIT_NEON
    return A / math.sqrt(1.0 + EN_Td / x0)


def n_gas(p_torr: float, T_gas: float = 300.0) -> float:
    return p_torr * TORR / (KB * T_gas)


def transport(gas: str = "neon", EN_Td: Sequence[float] | None = None, eps_max_eV: float = 400.0,
              n_grid: int = 1200) -> List[dict]:
    """Two-term transport records on a log grid of reduced fields, 2-1000 Td (increasing Te)."""
    ens = np.geomspace(2.0, 1000.0, 80) if EN_Td is None else np.asarray(EN_Td, float)
    xs = w.neon_xsecs() if gas == "neon" else w.argon_xsecs()
    mass = w.AMU_NE if gas == "neon" else w.AMU_AR
    recs = two_term(xs, mass, ens, eps_max_eV, n_grid)
    te = [2.0 / 3.0 * r["mean_eps_eV"] for r in recs]
    keep = [k for k in range(len(recs)) if k == 0 or te[k] > max(te[:k])]
    return [recs[k] for k in keep]


class Table:
    """Linear interpolation of the transport records in Te (as in the fluid kernel)."""

    def __init__(self, records):
        self.Te = np.array([2.0 / 3.0 * r["mean_eps_eV"] for r in records])
        self.q = {k: np.array([r[k] for r in records]) for k in records[0]}

    @classmethod
    def uniform(cls, records, n_T: int) -> "Table":
        """The records resampled (linear in Te) onto n_T uniform Te points: the table the fluid
        kernel interpolates (pic_fluid_init), so that derivatives match its slopes."""
        Te = np.array([2.0 / 3.0 * r["mean_eps_eV"] for r in records])
        grid = np.linspace(Te[0], Te[-1], n_T)
        keys = [k for k in records[0] if k != "mean_eps_eV"]
        out = [dict(mean_eps_eV=1.5 * x) for x in grid]
        for k in keys:
            v = np.interp(grid, Te, np.array([r[k] for r in records]))
            for d, x in zip(out, v):
                d[k] = float(x)
        return cls(out)

    def at(self, key, T):
        return np.interp(T, self.Te, self.q[key])

    def slope(self, key, T, h=1e-3):
        return (self.at(key, T + h) - self.at(key, T - h)) / (2 * h)

    def root(self, f):
        """Smallest Te of the table where f changes sign (linear interpolation)."""
        v = np.array([f(t) for t in self.Te])
        k = np.nonzero(np.sign(v[:-1]) != np.sign(v[1:]))[0]
        if len(k) == 0:
            return math.nan
        k = k[0]
        lo, hi = self.Te[k], self.Te[k + 1]
        for _ in range(60):
            mid = 0.5 * (lo + hi)
            if np.sign(f(mid)) == np.sign(f(lo)):
                lo = mid
            else:
                hi = mid
        return 0.5 * (lo + hi)


@dataclass
class Homogeneous:
    p_torr: float
    N_gas: float
    T0: float
    E0: float
    nu_w: float
    n0: float
    Gamma_T: float
    mu_e: float
    mu_i: float
    D_e: float
    R_m: float = math.nan
    I_A: float = math.nan


def homogeneous_E0(tab: Table, E0_over_p: float, p_torr: float = 1.0, n0: float = 1e15,
                   mu_iN: float | None = None, T_gas: float = 300.0) -> Homogeneous:
    """Imposed field E0 (V/cm/Torr x p): power balance mu_e(T0) E0^2 = L(T0) fixes T0;
    the wall loss equals the ionization frequency (pair-loss column).  mu_iN: the ion
    mobility x N (default: the neon fit at E0/N)."""
    N = n_gas(p_torr, T_gas)
    E0 = E0_over_p * 100.0 * p_torr
    if mu_iN is None:
        mu_iN = mu_iN_neon(E0 / N / 1e-21)
    T0 = tab.root(lambda T: tab.at("muN", T) / N * E0 * E0 - tab.at("lossN", T) * N)
    mu_e = tab.at("muN", T0) / N
    mu_i = mu_iN / N
    nu_w = tab.at("nu_izN", T0) * N
    return Homogeneous(p_torr, N, T0, E0, nu_w, n0, n0 * (mu_e + mu_i) * E0, mu_e, mu_i, tab.at("DN", T0) / N)


def homogeneous_R(tab: Table, pR_torr_cm: float, I_over_R: float, R_m: float = 0.01,
                  mu_iN: float | None = None, T_gas: float = 300.0) -> Homogeneous:
    """Tube of radius R, current I: nu_i(T0) = D_a(T0) (2.405/R)^2 (eq. 2) fixes T0, the power
    balance fixes E0, the current density J = I/(pi R^2) fixes n0 = (J/e)/((mu_e + mu_i) E0).
    mu_iN: the ion mobility x N (default: the neon fit at the state's E0/N)."""
    p = pR_torr_cm / (R_m * 100.0)
    N = n_gas(p, T_gas)
    g = (2.405 / R_m) ** 2

    def E_of(T):
        return math.sqrt(tab.at("lossN", T) * N / (tab.at("muN", T) / N))

    def mui(T):
        return (mu_iN if mu_iN is not None else mu_iN_neon(E_of(T) / N / 1e-21)) / N

    def f(T):
        Da = mui(T) * tab.at("DN", T) / tab.at("muN", T)
        return tab.at("nu_izN", T) * N - Da * g

    T0 = tab.root(f)
    mu_i = mui(T0)
    mu_e = tab.at("muN", T0) / N
    E0 = E_of(T0)
    nu_w = tab.at("nu_izN", T0) * N
    I = I_over_R * R_m
    GT = I / (math.pi * R_m * R_m) / QE
    n0 = GT / ((mu_e + mu_i) * E0)
    return Homogeneous(p, N, T0, E0, nu_w, n0, GT, mu_e, mu_i, tab.at("DN", T0) / N, R_m, I)


def linear(tab: Table, h: Homogeneous) -> dict:
    """Eqs. (19)-(23) at the homogeneous state h."""
    N, T0 = h.N_gas, h.T0
    De = lambda T: tab.at("DN", T) / N
    mue = lambda T: tab.at("muN", T) / N
    G = lambda T: 1.5 * T * tab.at("DeN", T) / N
    beta_e = lambda T: 1.5 * T * tab.at("mueN", T) / N
    d = 1e-3
    dG = (G(T0 + d) - G(T0 - d)) / (2 * d)
    dDe = (De(T0 + d) - De(T0 - d)) / (2 * d)
    K = dG - beta_e(T0) / mue(T0) * dDe                   # kappa_e0 / n0 (eq. 15)
    chi = G(T0) - beta_e(T0) / mue(T0) * De(T0)           # eq. 16
    nup = tab.slope("nu_izN", T0) * N
    L0 = tab.at("lossN", T0) * N
    Lp = tab.slope("lossN", T0) * N
    Da = h.mu_i * De(T0) / mue(T0)
    al, be, de = chi * nup / (Da * K), Lp / K, 2 * L0 * nup / (Da * K)
    disc = de - al * be
    out = dict(chi=chi, K=K, nu_p=nup, L0=L0, L_p=Lp, D_a=Da,
               chi_crit=(-(Da * Lp + math.sqrt(max(8 * Da * K * L0 * nup, 0.0))) / nup) if nup != 0 else math.nan)
    if disc <= 0 or -be + math.sqrt(disc) <= 0:
        out.update(gamma_max=math.nan, k_max=math.nan, lam=math.nan, v_ph=math.nan, unstable=False)
        return out
    k2 = -be + math.sqrt(disc)
    k = math.sqrt(k2)
    om = k * nup * h.E0 * De(T0) / (k2 * K + Lp)
    gmax = Da * (be - al - 2 * math.sqrt(disc))
    out.update(gamma_max=gmax, k_max=k, lam=2 * math.pi / k, v_ph=om / k, unstable=gmax > 0)
    return out


def gamma_k(tab: Table, h: Homogeneous, k: float) -> tuple[float, float]:
    """(gamma, omega) of wave number k from eqs. (19)-(20)."""
    lin = linear(tab, h)
    K, nup, Lp, L0, Da, chi = lin["K"], lin["nu_p"], lin["L_p"], lin["L0"], lin["D_a"], lin["chi"]
    den = k * k * K + Lp
    om = k * nup * h.E0 * h.D_e / den
    g = -Da * k * k - nup * (2 * L0 + chi * k * k) / den
    return g, om


def dispersion(tab: Table, h: Homogeneous, k: float, vector: bool = False):
    """(gamma, omega) of wave number k from the full linearisation of the fluid model as it is
    integrated (eqs. 3-5 with the flux of eq. 11, the field of eqs. 10 + 12 and the energy flux
    of eqs. 8-9 read as beta = 3/2 Te mu_eps, G = 3/2 Te D_eps; fixed nu_w = nu_i(T0)), keeping
    what eq. (18) drops: the time
    derivative of the energy equation, the temperature terms of the field and of the fluxes.
    Perturbations (dn, dT) exp(i k x - i Omega t) solve -i Omega M v = A v with
    M = [[1, 0], [3/2 T0, 3/2 n0]]; the root with the largest growth rate is returned, and with
    vector=True also its eigenvector (dn, dT)."""
    N, T0, n0, GT = h.N_gas, h.T0, h.n0, h.Gamma_T
    d = 1e-4
    mu = lambda T: tab.at("muN", T) / N
    D = lambda T: tab.at("DN", T) / N
    mue = lambda T: tab.at("mueN", T) / N
    De = lambda T: tab.at("DeN", T) / N
    der = lambda F: (F(T0 + d) - F(T0 - d)) / (2 * d)
    mui = h.mu_i
    a = lambda T: mui / (mu(T) + mui)
    a0, ap = a(T0), der(a)
    D0, Dp = D(T0), der(D)
    mu0, mup = mu(T0), der(mu)

    E0 = GT / (n0 * (mu0 + mui))
    Gam0 = -(1.0 - a0) * GT
    me0, mep, De0, Dep = mue(T0), der(mue), De(T0), der(De)
    L0 = tab.at("lossN", T0) * N
    Lp = tab.slope("lossN", T0) * N
    nup = tab.slope("nu_izN", T0) * N
    ik = 1j * k
    # continuity: Gamma = -a d_x(n D) - (1 - a) Gamma_T, source n (nu_i - nu_w)
    A11 = -a0 * k * k * D0
    A12 = -a0 * k * k * n0 * Dp - ik * ap * GT + n0 * nup
    # field (eq. 17) and fluxes
    # E = -d_x(n D)/(n mu) + Gamma_T/(n (mu + mu_i))
    dE_dn = -ik * D0 / (n0 * mu0) - E0 / n0
    dE_dT = -ik * Dp / mu0 - E0 * mup / (mu0 + mui)
    dG_dn = -a0 * ik * D0
    dG_dT = -a0 * ik * n0 * Dp + ap * GT
    dH_dn = -1.5 * (me0 * dE_dn * n0 * T0 + me0 * E0 * T0) - 1.5 * ik * De0 * T0
    dH_dT = -1.5 * (mep * E0 * n0 * T0 + me0 * dE_dT * n0 * T0 + me0 * E0 * n0) - 1.5 * ik * n0 * (De0 + Dep * T0)
    dP_dn = -(dG_dn * E0 + Gam0 * dE_dn)
    dP_dT = -(dG_dT * E0 + Gam0 * dE_dT)
    B1 = -ik * dH_dn + dP_dn - L0
    B2 = -ik * dH_dT + dP_dT - n0 * Lp
    M = np.array([[1.0, 0.0], [1.5 * T0, 1.5 * n0]], complex)
    A = np.array([[A11, A12], [B1, B2]], complex)
    lam, vec = np.linalg.eig(np.linalg.solve(M, A))
    W = lam / (-1j)
    i = int(np.argmax(W.imag))
    if vector:
        return float(W[i].imag), float(W[i].real), vec[:, i]
    return float(W[i].imag), float(W[i].real)


def dispersion_max(tab: Table, h: Homogeneous, L: float, m_max: int = 256) -> dict:
    """Fastest-growing mode m = 1..m_max of a periodic column of length L (full linearisation)."""
    best = max(range(1, m_max + 1), key=lambda m: dispersion(tab, h, 2 * math.pi * m / L)[0])
    k = 2 * math.pi * best / L
    g, om = dispersion(tab, h, k)
    return dict(m=best, lam=L / best, gamma=g, v_ph=om / k)


def potential_drop(E_nodes: np.ndarray, dx: float, cells: int, start: int = 0) -> float:
    """Potential drop over `cells` consecutive cells of a periodic column from the total node
    field E = -E0 + E_sp (eq. 1: over one striation it equals E0 lambda, the space-charge field
    averaging to zero over a period): |-sum_j E_j dx| over nodes start .. start + cells - 1."""
    idx = (start + np.arange(cells)) % len(E_nodes)
    return float(abs(-np.sum(E_nodes[idx]) * dx))


def observables(t: np.ndarray, modes: np.ndarray, L: float) -> dict:
    """Striation observables from a record of modes: t (snapshot times, increasing),
    modes [snap, 1 + M] complex with entry 0 the mean density."""
    mean = modes[:, 0].real
    A = np.abs(modes[:, 1:]) / mean[:, None]
    sat = t >= 0.5 * t[-1]
    power = (A[sat] ** 2).mean(0)
    m = int(np.argmax(power)) + 1
    k = 2 * math.pi * m / L
    ts = t[sat]
    ph = np.unwrap(np.angle(modes[sat, m]))
    v_ph = -np.polyfit(ts, ph, 1)[0] / k if len(ts) >= 3 else math.nan
    a = A[:, m - 1]
    a_sat = math.sqrt(power[m - 1])
    a0 = max(a[0], 1e-30)
    grow = np.nonzero((a > 10 * a0) & (a < 0.1 * a_sat))[0]
    gamma = math.nan
    if len(grow) >= 3:
        i0, i1 = grow[0], grow[-1]
        if i1 - i0 >= 2:
            gamma = np.polyfit(t[i0:i1 + 1], np.log(a[i0:i1 + 1]), 1)[0]
    return dict(m=m, lam=L / m, v_ph=v_ph, gamma=gamma, amp_sat=a_sat, amp0=a[0])


def initial_state(N: int, h: Homogeneous, seed: int, amp: float = 1e-3):
    """Homogeneous state with a seeded white perturbation of relative amplitude amp."""
    rng = np.random.default_rng(seed)
    n = h.n0 * (1.0 + amp * rng.standard_normal(N))
    T = np.full(N, h.T0)
    return n, T


def fluid_columns(states: Sequence[Homogeneous], L_m: float, n_cells: int, pair: bool = True) -> List[dict]:
    """Fluid columns of the homogeneous states.  pair=True (default): losses equal to the
    ionization of the column at every step (the particle model's pair removal; a fixed nu_w
    lets the mean density run away once striations change the mean ionization); pair=False:
    nu_w fixed at the homogeneous value (eq. 3 as written; used for the linear phase)."""
    from . import FLUID_LOSS_FIXED, FLUID_LOSS_PAIR
    return [dict(L_m=L_m, N_gas_m3=h.N_gas, mu_iN=h.mu_i * h.N_gas, Gamma_T=h.Gamma_T, nu_w=h.nu_w,
                 n_cells=n_cells, loss=FLUID_LOSS_PAIR if pair else FLUID_LOSS_FIXED) for h in states]


def fluid_screen(records, states: Sequence[Homogeneous], L_m: float = 0.30, n_cells: int = 4096,
                 dt: float = 2e-9, steps: int = 20000, diag_every: int = 100, n_modes: int = 64,
                 seed: int = 11, n_T: int = 128, closure=None) -> dict:
    """Advance one fluid column per state for `steps` steps; return the observables per
    column, the device time and the number of kernel launches."""
    f = Fluid(fluid_columns(states, L_m, n_cells), records, n_T=n_T, dt_s=dt, diag_every=diag_every,
              n_modes=n_modes)
    if closure is not None:
        f.set_closure(*closure)
    for k, h in enumerate(states):
        f.set_state(k, *initial_state(n_cells, h, seed + k))
    f.step(steps)
    ms, launches = f.elapsed()
    rec = f.modes()
    t = (np.arange(rec.shape[0]) + 1) * diag_every * dt
    obs = [observables(t, rec[:, k], L_m) for k in range(len(states))]
    f.close()
    return dict(obs=obs, ms=ms, launches=launches, t=t, modes=rec)


def pic_columns(E0_over_p: Sequence[float], p_torr: float = 1.0, L_m: float = 0.10, n_cells: int = 2048,
                particles: int = 1_000_000, n0: float = 1e15, seed: int = 21, gas: str = "neon"):
    """Particle-model columns (pair losses, imposed field) at the given reduced fields."""
    base = w.config_neon_column(n_per_species=particles) if gas == "neon" else w.config_argon_small()
    return [base.with_(pressure_torr=p_torr, L_m=L_m, n_cells=n_cells, E0_Vpm=e * 100.0 * p_torr,
                       drive=w.DRIVE_E0, n0_m3=n0, n_e0=particles, n_i0=particles, loss_mode=w.LOSS_PAIR,
                       diag_every=50, sort_every=1000, seed=seed + k, column=k)
            for k, e in enumerate(E0_over_p)]


def pic_record(params, windows: int, window: int):
    """Run the columns as one GPU batch; per window and column: the density modes (FFT of
    the window-averaged n_e), the ion mobility x N from the window's ion flux, and the
    device time of the whole run."""
    from . import Batch
    b = Batch(params)
    for c in b.columns:
        c.moments(reset=True)
    M = 64
    rec = np.zeros((windows, len(params), M + 1), complex)
    mob = np.zeros((windows, len(params)))
    import time
    t0 = time.perf_counter()
    for s in range(windows):
        b.step(window)
        for k, (c, p) in enumerate(zip(b.columns, params)):
            m = c.moments(reset=True)
            ne = m["n_e"]
            F = np.fft.fft(ne) / len(ne)
            rec[s, k, 0] = ne.mean()
            rec[s, k, 1:] = F[1:M + 1]
            # the applied field points along -x in the particle model: ions drift towards -x
            mob[s, k] = abs(m["gamma_i"].sum()) / max(m["n_i"].sum(), 1e-30) / p.E0_Vpm * n_gas(p.pressure_torr)
    wall = time.perf_counter() - t0
    b.close()
    return rec, mob, wall


def compare(E0_over_p: Sequence[float], p_torr: float = 1.0, L_m: float = 0.10, pic_cells: int = 2048,
            fluid_cells: int = 2048, particles: int = 1_000_000, windows: int = 50, window: int = 20000,
            fluid_dt: float = 2e-8, fluid_diag: int = 40, mu_iN: float | None = None, records=None,
            closure=None, on_pic=None) -> dict:
    """Particle model and fluid model at the same imposed reduced fields: striation
    observables of both and the time each took per condition."""
    records = records or transport()
    tab = Table(records)
    params = pic_columns(E0_over_p, p_torr, L_m, pic_cells, particles)
    rec, mob, wall = pic_record(params, windows, window)
    if on_pic is not None:
        on_pic(rec, mob, wall)
    dt_pic = params[0].dt_s
    t_pic = (np.arange(windows) + 0.5) * window * dt_pic
    pic_obs = [observables(t_pic, rec[:, k], L_m) for k in range(len(params))]
    mu_meas = float(np.median(mob[windows // 2:])) if mu_iN is None else mu_iN
    states = [homogeneous_E0(tab, e, p_torr, mu_iN=mu_meas) for e in E0_over_p]
    T_total = windows * window * dt_pic
    steps = int(round(T_total / fluid_dt))
    fl = fluid_screen(records, states, L_m=L_m, n_cells=fluid_cells, dt=fluid_dt, steps=steps,
                      diag_every=fluid_diag, closure=closure)
    lin = [linear(tab, h) for h in states]
    return dict(E0_over_p=list(E0_over_p), pic=pic_obs, fluid=fl["obs"], linear=lin, mu_iN=mu_meas,
                pic_seconds=wall, fluid_ms=fl["ms"], simulated_s=T_total, fluid_steps=steps,
                pic_steps=windows * window, pic_modes=rec, fluid_modes=fl["modes"], t_pic=t_pic, t_fluid=fl["t"])


def coarsen(m: dict, f: int) -> dict:
    """A moment window averaged over blocks of f nodes: densities, fluxes, rates and the field as
    block means, the mean energy weighted by the electron density."""
    if f == 1:
        return m
    out = {}
    for k, v in m.items():
        if not isinstance(v, np.ndarray):
            out[k] = v
            continue
        out[k] = v.reshape(-1, f).mean(1)
    ne = m["n_e"].reshape(-1, f)
    out["mean_eps_e"] = (m["mean_eps_e"].reshape(-1, f) * ne).sum(1) / np.maximum(ne.sum(1), 1e-300)
    return out


def _cathode_v(v_ph: float, frame: str) -> float:
    """Phase velocity counted positive towards the cathode: the particle model's field
    points along -x (cathode at -x), the fluid model's along +x."""
    return -v_ph if frame == "pic" else v_ph


def study(E_compare: Sequence[float], E_train: Sequence[float], p_torr: float = 1.0, L_m: float = 0.10,
          n_cells: int = 2048, particles: int = 1_000_000, windows: int = 200, window: int = 4000,
          early: int = 100, early_window: int = 1000, agg: int = 4, fluid_dt: float = 2e-9, fluid_diag: int = 20,
          train_steps: int = 3000, batch: int = 8192, lr: float = 1e-3, period: int = 10,
          components=((0.0, 1.0, 1.0), (0.0, 0.0, 1.0)), nu_bound: float = 1.0, stencils=(1,), seed: int = 7,
          fluid_cells: int | None = None, save: str | None = None, load: str | None = None,
          log=print) -> dict:
    """Particle model (one GPU batch: comparison and training fields), closure training on
    its moment windows, fluid model with and without the trained closure at the comparison
    fields; striation observables, closure gain and times.  The particle record takes
    `early` windows of `early_window` steps (growth phase), then `windows` windows of
    `window` steps; closure data come from the long windows, `agg` at a time.
    components: which network outputs the fluid screen applies (flux, energy flux,
    ionization), one triple or a list of triples (each closure is then run with each; the
    first of the first stencil is the study's main closure); the flux corrections enter the
    fluid step implicitly (upwind advection), positivity-preserving at any time step.
    fluid_cells: cells of the fluid columns (default: those of the particle columns); with fewer,
    the particle model's moment windows are averaged onto the fluid grid (blocks of
    n_cells / fluid_cells cells; the mean energy weighted by density) before the closure samples
    are formed, so that the network sees the fluid model's resolution."""
    import time
    import torch
    from . import Batch, Mlp
    from . import closure as cl
    fluid_cells = fluid_cells or n_cells
    if n_cells % fluid_cells:
        raise ValueError("the particle cells must be a multiple of the fluid cells")
    records = transport()
    tab = Table(records)
    Es = list(E_compare) + list(E_train)
    params = pic_columns(Es, p_torr, L_m, n_cells, particles)
    ncmp = len(E_compare)
    M = 64
    fs = cl.FEATURE_SCALE
    if load is not None:
        # the particle record and the trained closures of an earlier run of the same study
        z = np.load(load)
        meta = json.loads(str(z["meta"]))
        mine = dict(E_compare=list(E_compare), E_train=list(E_train), p_torr=p_torr, L_m=L_m, n_cells=n_cells,
                    fluid_cells=fluid_cells, particles=particles, stencils=list(stencils), seed=seed)
        if any(meta[k] != v for k, v in mine.items()):
            raise ValueError(f"{load} holds another study: {meta}")
        rec, t_pic, mu = z["rec"], z["t_pic"], [float(v) for v in z["mu"]]
        total_steps, dt_pic, pic_run, held = meta["total_steps"], meta["dt_pic"], meta["pic_run"], meta["held"]
        nets = []
        for k, st_k in enumerate(meta["stencils"]):
            net = Mlp(seed=seed)
            net.set_params(z["net_params"][k])
            nets.append(dict(stencil=st_k, net=net, ts=z["net_ts"][k], mse_net=z["net_mse"][k],
                             mse_tab=z["net_mse_tab"][k], train_s=float(z["net_train_s"][k]),
                             last=float(z["net_last"][k]), n=int(z["net_n"][k])))
        log(f"particle record and {len(nets)} closures from {load}")
    else:
        b = Batch(params)
        for c in b.columns:
            c.moments(reset=True)
        plan = [early_window] * early + [window] * windows
        nw = len(plan)
        rec = np.zeros((nw, len(Es), M + 1), complex)
        mob = np.zeros((nw, len(Es)))
        acc = [dict() for _ in Es]
        train_windows = [[] for _ in Es]
        keys = ("n_e", "mean_eps_e", "gamma_e", "heat_e", "iz_rate", "gamma_i", "E")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pic_run = 0.0
        for s, steps_s in enumerate(plan):
            ta = time.perf_counter()
            b.step(steps_s)
            pic_run += time.perf_counter() - ta
            for k, (c, p) in enumerate(zip(b.columns, params)):
                m = c.moments(reset=True)
                rec[s, k, 0] = m["n_e"].mean()
                rec[s, k, 1:] = (np.fft.fft(m["n_e"]) / n_cells)[1:M + 1]
                mob[s, k] = abs(m["gamma_i"].sum()) / max(m["n_i"].sum(), 1e-30) / p.E0_Vpm * n_gas(p_torr)
                if k >= ncmp and s >= early:
                    for q in keys:
                        acc[k][q] = acc[k].get(q, 0.0) + m[q] / agg
                    if (s - early + 1) % agg == 0:
                        train_windows[k].append(acc[k])
                        acc[k] = dict()
        wall = time.perf_counter() - t0
        b.close()
        total_steps = int(sum(plan))
        log(f"particle batch: {len(Es)} columns, {total_steps} steps, {pic_run:.1f} s stepping, {wall:.1f} s total")
        dt_pic = params[0].dt_s
        ends = np.cumsum(plan)
        t_pic = (ends - 0.5 * np.array(plan)) * dt_pic
        amp = np.abs(rec[:, :, 1:]).max(2) / rec[:, :, 0].real
        mu = []
        for k in range(len(Es)):
            # ion mobility of the uniform column: windows after the first 0.2 us, before striations
            sel = [s for s in range(nw) if t_pic[s] > 2e-7 and amp[s, k] < 0.05][:8] or [min(nw - 1, early)]
            mu.append(float(np.median(mob[sel, k])))
        # closure data from the training columns: residuals of the tabulated closure, one network per
        # stencil spacing (the first is the study's main closure)
        T_range = (tab.Te[0], tab.Te[-1])
        held = ncmp + (len(E_train) // 2)                  # one training column held out (split by run)
        nets = []
        for st_k in stencils:
            Xs, Ys, col_of = [], [], []
            for k in range(ncmp, len(Es)):
                for m in train_windows[k][2:]:
                    X, Y = cl.residual_samples(coarsen(m, n_cells // fluid_cells), params[k], tab, mu[k], T_range,
                                               step=st_k)
                    Xs.append(X)
                    Ys.append(Y)
                    col_of.append(np.full(len(X), k))
            X = np.concatenate(Xs)
            Y = np.concatenate(Ys)
            col_of = np.concatenate(col_of)
            ts = np.maximum(np.std(Y, 0), 1e-30).astype(np.float32)
            tr, te = col_of != held, col_of == held
            Xn, Yn = (X / fs).astype(np.float32), (Y / ts).astype(np.float32)
            rng = np.random.default_rng(seed)
            perm = rng.permutation(np.nonzero(tr)[0])
            Xd = torch.from_numpy(Xn[perm]).cuda()
            Yd = torch.from_numpy(Yn[perm]).cuda()
            net = Mlp(seed=seed)
            torch.cuda.synchronize()
            ta = time.perf_counter()
            last = net.train(Xd, Yd, batch=batch, steps=train_steps, lr=lr)
            torch.cuda.synchronize()
            train_s = time.perf_counter() - ta
            Yh = net.forward(torch.from_numpy(Xn[te]).cuda()).cpu().numpy()
            mse_net = ((Yh - Yn[te]) ** 2).mean(0)
            mse_tab = (Yn[te] ** 2).mean(0)             # the tabulated closure alone predicts zero residual
            log(f"closure (stencil {st_k}): {len(X)} samples, held-out column E0/p = {Es[held]}, "
                f"mse net {mse_net} vs table {mse_tab}")
            nets.append(dict(stencil=st_k, net=net, ts=ts, mse_net=mse_net, mse_tab=mse_tab, train_s=train_s,
                             last=last, n=len(X)))
        if save is not None:
            meta = dict(E_compare=list(E_compare), E_train=list(E_train), p_torr=p_torr, L_m=L_m, n_cells=n_cells,
                        fluid_cells=fluid_cells, particles=particles, stencils=list(stencils), seed=seed,
                        total_steps=total_steps, dt_pic=dt_pic, pic_run=pic_run, held=held)
            np.savez(save, meta=json.dumps(meta), rec=rec, t_pic=t_pic, mu=np.array(mu),
                     net_params=np.stack([d["net"].params() for d in nets]),
                     net_ts=np.stack([d["ts"] for d in nets]), net_mse=np.stack([d["mse_net"] for d in nets]),
                     net_mse_tab=np.stack([d["mse_tab"] for d in nets]),
                     net_train_s=np.array([d["train_s"] for d in nets]),
                     net_last=np.array([d["last"] for d in nets]), net_n=np.array([d["n"] for d in nets]))
    net, ts, mse_net, mse_tab, train_s, last = (nets[0][k] for k in ("net", "ts", "mse_net", "mse_tab",
                                                                    "train_s", "last"))
    # fluid model at the comparison fields, same simulated time, noise of the particle model
    states = [homogeneous_E0(tab, e, p_torr, mu_iN=mu[k]) for k, e in enumerate(E_compare)]
    steps = int(round(total_steps * dt_pic / fluid_dt))
    diag = fluid_diag
    noise = 1.0 / math.sqrt(particles / fluid_cells)
    masks = np.atleast_2d(np.asarray(components, np.float32))
    out = {}
    vname = lambda i, d, mi: ("fluid_closure" if i == 0 and mi == 0
                              else f"fluid_closure_s{d['stencil']}_c{'_'.join(f'{v:g}' for v in masks[mi])}")
    variants = [("fluid", True, None)] + [
        (vname(i, d, mi), True, (d["net"], period, fs, d["ts"] * masks[mi], nu_bound, d["stencil"]))
        for i, d in enumerate(nets) for mi in range(len(masks))]
    for name, pair, clo in variants:
        f = Fluid(fluid_columns(states, L_m, fluid_cells, pair=pair), records, n_T=128, dt_s=fluid_dt,
                  diag_every=diag, n_modes=M)
        if clo is not None:
            f.set_closure(*clo)
        for k, h in enumerate(states):
            f.set_state(k, *initial_state(fluid_cells, h, seed + 100 + k, amp=noise))
        f.step(steps)
        ms, launches = f.elapsed()
        r = f.modes()
        f.close()
        t = (np.arange(r.shape[0]) + 1) * diag * fluid_dt
        obs = [observables(t, r[:, k], L_m) for k in range(ncmp)]
        for o in obs:
            o["v_ph"] = _cathode_v(o["v_ph"], "fluid")
        out[name] = dict(obs=obs, ms=ms, launches=launches, modes=r, t=t)
        log(f"{name}: {steps} steps of {ncmp} columns in {ms:.1f} ms ({launches} launches)")
    pic_obs = [observables(t_pic, rec[:, k], L_m) for k in range(ncmp)]
    for o in pic_obs:
        o["v_ph"] = _cathode_v(o["v_ph"], "pic")
    lin = [linear(tab, h) for h in states]
    full = [dispersion_max(tab, h, L_m) for h in states]
    pic_per_col = pic_run / len(Es)
    return dict(E_compare=list(E_compare), E_train=list(E_train), mu_iN=mu, pic=pic_obs,
                fluid=out["fluid"]["obs"], fluid_closure=out["fluid_closure"]["obs"], linear=lin,
                dispersion=full,
                pic_seconds_per_column=pic_per_col,
                fluid_seconds_per_column=out["fluid"]["ms"] / 1e3 / ncmp,
                fluid_closure_seconds_per_column=out["fluid_closure"]["ms"] / 1e3 / ncmp,
                simulated_s=total_steps * dt_pic, train_seconds=train_s, train_loss=last,
                components=masks.tolist(),
                stencils=list(stencils), nu_bound=nu_bound,
                closures=[dict(stencil=d["stencil"], components=masks[mi].tolist(), mse_net=d["mse_net"].tolist(),
                               mse_table=d["mse_tab"].tolist(),
                               lam=[o["lam"] for o in out[vname(i, d, mi)]["obs"]],
                               v_ph=[o["v_ph"] for o in out[vname(i, d, mi)]["obs"]],
                               gamma=[o["gamma"] for o in out[vname(i, d, mi)]["obs"]],
                               amp_sat=[o["amp_sat"] for o in out[vname(i, d, mi)]["obs"]])
                          for i, d in enumerate(nets) for mi in range(len(masks))],
                n_samples=int(nets[0]["n"]), held_out_E=Es[held], mse_net=mse_net.tolist(), mse_table=mse_tab.tolist(),
                target_scale=ts.tolist(), pic_modes=rec, t_pic=t_pic,
                fluid_modes=out["fluid"]["modes"], fluid_closure_modes=out["fluid_closure"]["modes"],
                t_fluid=out["fluid"]["t"])


GRID_PR = np.geomspace(0.3, 3.0, 32)     # pR of the fluid screen, Torr cm
GRID_IR = np.geomspace(0.01, 1.0, 32)    # I/R of the fluid screen, A/m


def grid_points(idx: Sequence[int] = (4, 12, 20, 28)) -> list:
    """Sampled points of the 32 x 32 (pR, I/R) screen: the sub-grid idx x idx (16 points)."""
    return [(float(GRID_PR[i]), float(GRID_IR[j])) for i in idx for j in idx]


def grid_study(points, load: str | None = None, R_m: float = 0.01, L_m: float = 0.30, n_cells: int = 16384,
               fluid_cells: int = 4096, particles: int = 1_000_000, dt: float = 1.6e-11,
               simulated_s: float = 3.6e-5, windows: int = 300, early: int = 100, early_frac: float = 0.1,
               diag_every: int = 120, fluid_dt: float = 2e-9, fluid_diag: int = 20, period: int = 10,
               components=((0.0, 1.0, 1.0), (0.0, 0.0, 1.0)), nu_bound: float = 0.5, stencils=(1, 16),
               agg: int = 2, train_steps: int = 3000, batch: int = 8192, lr: float = 1e-3, seed: int = 7,
               log=print) -> dict:
    """The particle model at (pR, I/R) points of a tube of radius R (current drive: eq. 2 gives the
    homogeneous field and density), one GPU batch, against the fluid screen at the same points
    (homogeneous states of eq. 2, pair losses, each column with the ion mobility measured in its
    particle column) with and without a learned closure, over the same simulated time.
    Closures: with `load` (the .npz that study(save=...) writes) the networks of that study;
    without it, two-fold cross-validation over the points: the points split by the parity of
    their index sum on the 4 x 4 sub-grid (a checkerboard), one network per fold and stencil
    trained on the moment windows of the other fold's columns and applied to this fold's.
    dt is common to the batch and must keep nu* dt <= 0.3 at the highest pressure.  The record
    takes `early` windows covering early_frac of the time (growth), then `windows` windows; the
    closure data come from the long windows, `agg` at a time."""
    import time
    import torch
    from . import Batch, Mlp, drive_ri
    from . import closure as cl
    records = transport()
    tab = Table(records)
    total = int(round(simulated_s / dt))
    ew = max(1, int(total * early_frac / early) // diag_every * diag_every)
    lw = max(1, int((total - early * ew) / windows) // diag_every * diag_every)
    plan = [ew] * early + [lw] * windows
    base = w.config_neon_column(n_per_species=particles)
    params = [base.with_(pressure_torr=pr / (R_m * 100.0), R_m=R_m, I_A=ir * R_m, L_m=L_m, n_cells=n_cells,
                         dt_s=dt, drive=w.DRIVE_RI, n_e0=particles, n_i0=particles, loss_mode=w.LOSS_PAIR,
                         diag_every=diag_every, sort_every=1000, seed=seed + 40 + k, column=k)
              for k, (pr, ir) in enumerate(points)]
    drives = [drive_ri(p) for p in params]   # eq. 2 as the library resolves it: E0, n0, Te0, mu_i N
    b = Batch(params)
    for c in b.columns:
        c.moments(reset=True)
    M = 64
    nw = len(plan)
    npt = len(points)
    rec = np.zeros((nw, npt, M + 1), complex)
    mob = np.zeros((nw, npt))
    keys = ("n_e", "mean_eps_e", "gamma_e", "heat_e", "iz_rate", "gamma_i", "E")
    acc = [dict() for _ in points]
    train_windows = [[] for _ in points]
    torch.cuda.synchronize()
    pic_run = 0.0
    for s_, steps_s in enumerate(plan):
        ta = time.perf_counter()
        b.step(steps_s)
        pic_run += time.perf_counter() - ta
        for k, c in enumerate(b.columns):
            m = c.moments(reset=True)
            rec[s_, k, 0] = m["n_e"].mean()
            rec[s_, k, 1:] = (np.fft.fft(m["n_e"]) / n_cells)[1:M + 1]
            mob[s_, k] = abs(m["gamma_i"].sum()) / max(m["n_i"].sum(), 1e-30) / drives[k]["E0_Vpm"] * \
                n_gas(params[k].pressure_torr)
            if load is None and s_ >= early:
                for q in keys:
                    acc[k][q] = acc[k].get(q, 0.0) + m[q] / agg
                if (s_ - early + 1) % agg == 0:
                    train_windows[k].append(acc[k])
                    acc[k] = dict()
    b.close()
    steps_total = int(sum(plan))
    log(f"particle batch: {npt} columns, {steps_total} steps, {pic_run:.1f} s stepping")
    ends = np.cumsum(plan)
    t_pic = (ends - 0.5 * np.array(plan)) * dt
    amp = np.abs(rec[:, :, 1:]).max(2) / rec[:, :, 0].real
    mu = []
    for k in range(npt):
        # ion mobility of the uniform column: windows after the first 0.2 us, before striations
        sel = [q for q in range(nw) if t_pic[q] > 2e-7 and amp[q, k] < 0.05][:8] or [min(nw - 1, early)]
        mu.append(float(np.median(mob[sel, k])))
    states = [homogeneous_R(tab, pr, ir, R_m=R_m, mu_iN=mu[k]) for k, (pr, ir) in enumerate(points)]
    fs = cl.FEATURE_SCALE
    # networks: nets[(fold, stencil)] = (net, target scale); fold of point k (its test fold)
    side = int(round(math.sqrt(npt)))
    fold = [((k // side) + (k % side)) % 2 for k in range(npt)] if load is None else [0] * npt
    nets, mse = {}, {}
    if load is not None:
        z = np.load(load)
        meta = json.loads(str(z["meta"]))
        for j, st_k in enumerate(meta["stencils"]):
            net = Mlp(seed=seed)
            net.set_params(z["net_params"][j])
            nets[(0, st_k)] = (net, z["net_ts"][j])
        stencils = tuple(meta["stencils"])
    else:
        T_range = (tab.Te[0], tab.Te[-1])
        for f_ in (0, 1):
            for st_k in stencils:
                Xs, Ys, test = [], [], []
                for k in range(npt):
                    for m in train_windows[k][2:]:
                        X, Y = cl.residual_samples(coarsen(m, n_cells // fluid_cells), params[k], tab, mu[k],
                                                   T_range, step=st_k)
                        Xs.append(X)
                        Ys.append(Y)
                        test.append(np.full(len(X), fold[k] == f_))
                X, Y, test = np.concatenate(Xs), np.concatenate(Ys), np.concatenate(test)
                tr = ~test
                ts = np.maximum(np.std(Y[tr], 0), 1e-30).astype(np.float32)
                Xn, Yn = (X / fs).astype(np.float32), (Y / ts).astype(np.float32)
                perm = np.random.default_rng(seed + f_).permutation(np.nonzero(tr)[0])
                net = Mlp(seed=seed)
                net.train(torch.from_numpy(Xn[perm]).cuda(), torch.from_numpy(Yn[perm]).cuda(), batch=batch,
                          steps=train_steps, lr=lr)
                Yh = net.forward(torch.from_numpy(Xn[test]).cuda()).cpu().numpy()
                mse[(f_, st_k)] = (((Yh - Yn[test]) ** 2).mean(0).tolist(), (Yn[test] ** 2).mean(0).tolist(),
                                   int(tr.sum()), int(test.sum()))
                nets[(f_, st_k)] = (net, ts)
                log(f"fold {f_} stencil {st_k}: {int(tr.sum())} training samples, held-out mse "
                    f"{mse[(f_, st_k)][0]} vs table {mse[(f_, st_k)][1]}")
    steps = int(round(steps_total * dt / fluid_dt))
    noise = 1.0 / math.sqrt(particles / fluid_cells)
    masks = np.atleast_2d(np.asarray(components, np.float32))
    ok = [math.isfinite(h.T0) for h in states]

    def fluid_obs(ks, clo):
        """observables of the fluid columns of points ks (homogeneous start), closure clo or none"""
        f = Fluid(fluid_columns([states[k] for k in ks], L_m, fluid_cells), records, n_T=128, dt_s=fluid_dt,
                  diag_every=fluid_diag, n_modes=M)
        if clo is not None:
            f.set_closure(*clo)
        for j, k in enumerate(ks):
            f.set_state(j, *initial_state(fluid_cells, states[k], seed + 100 + k, amp=noise))
        f.step(steps)
        ms, _ = f.elapsed()
        r = f.modes()
        f.close()
        t = (np.arange(r.shape[0]) + 1) * fluid_diag * fluid_dt
        obs = []
        for j in range(len(ks)):
            o = observables(t, r[:, j], L_m)
            o["v_ph"] = _cathode_v(o["v_ph"], "fluid")
            obs.append(o)
        return obs, ms

    variants, vms = {}, {}
    names = [("fluid", None, None)] + [(f"closure_s{st_k}_c{'_'.join(f'{v:g}' for v in masks[mi])}", st_k, mi)
                                      for st_k in stencils for mi in range(len(masks))]
    for name, st_k, mi in names:
        obs_all, ms_all = [None] * npt, 0.0
        for f_ in sorted(set(fold)):
            ks = [k for k in range(npt) if fold[k] == f_ and ok[k]]
            if not ks:
                continue
            clo = None
            if st_k is not None:
                net, ts = nets[(f_, st_k)]
                clo = (net, period, fs, ts * masks[mi], nu_bound, st_k)
            obs, ms = fluid_obs(ks, clo)
            for k, o in zip(ks, obs):
                obs_all[k] = o
            ms_all += ms
        variants[name] = obs_all
        vms[name] = ms_all
        log(f"{name}: {steps} steps of {sum(ok)} columns in {ms_all:.1f} ms")
    pic_obs = []
    for k in range(npt):
        o = observables(t_pic, rec[:, k], L_m)
        o["v_ph"] = _cathode_v(o["v_ph"], "pic")
        pic_obs.append(o)
    lin = [linear(tab, h) if g else None for h, g in zip(states, ok)]
    return dict(points=[list(p) for p in points], dt=dt, steps=steps_total, simulated_s=steps_total * dt,
                pic=pic_obs, pic_seconds_per_column=pic_run / npt, mu_iN=mu,
                pic_E0=[d["E0_Vpm"] for d in drives], pic_n0=[d["n0_m3"] for d in drives],
                pic_Te0=[d["Te0_eV"] for d in drives],
                fluid_T0=[h.T0 for h in states], fluid_E0=[h.E0 for h in states], fluid_n0=[h.n0 for h in states],
                linear=lin, variants=variants,
                fluid_seconds_per_column={k: v / 1e3 / max(1, sum(ok)) for k, v in vms.items()},
                closures="loaded from " + load if load else "two-fold cross-validation over the points",
                fold=fold, mse={f"fold{k[0]}_s{k[1]}": v for k, v in mse.items()})


def _jsonable(o):
    if isinstance(o, dict):
        return {k: _jsonable(v) for k, v in o.items() if not isinstance(v, np.ndarray)}
    if isinstance(o, (list, tuple)):
        return [_jsonable(v) for v in o]
    if isinstance(o, (np.floating, np.integer)):
        return o.item()
    if isinstance(o, np.bool_):
        return bool(o)
    return o


def main(argv=None) -> int:
    """python -m paper_2202_03215_gb300.screen study [--out FILE]: the particle/fluid study of
    neon at 1 Torr (L = 10 cm, 2048 cells, 1e6 particles per species, 36 us), fields
    6..20 V/cm/Torr compared, 7..21 for training; prints one line per field and writes JSON."""
    import argparse
    import json
    ap = argparse.ArgumentParser(prog="python -m paper_2202_03215_gb300.screen")
    ap.add_argument("what", choices=["study", "fluid", "grid"])
    ap.add_argument("--out", default=None)
    ap.add_argument("--nu-bound", type=float, default=0.5)
    ap.add_argument("--stencils", type=int, nargs="+", default=[1], help="closure stencil spacings, cells")
    ap.add_argument("--columns", type=int, default=152)
    ap.add_argument("--cells", type=int, default=4096)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--L", type=float, default=0.10, help="study: column length, m")
    ap.add_argument("--pic-cells", type=int, default=2048, help="study: cells of the particle and fluid columns")
    ap.add_argument("--particles", type=int, default=1_000_000, help="study: particles per species and column")
    ap.add_argument("--windows", type=int, default=200, help="study: long windows of the particle record")
    ap.add_argument("--window", type=int, default=4000, help="study: steps per long window")
    ap.add_argument("--agg", type=int, default=4, help="study: long windows averaged per closure sample window")
    ap.add_argument("--train-steps", type=int, default=3000)
    ap.add_argument("--fluid-cells", type=int, default=None, help="study: cells of the fluid columns")
    ap.add_argument("--early", type=int, default=100, help="study: growth-phase windows of 1000 steps")
    ap.add_argument("--components", nargs="+", default=["0,1,1", "0,0,1"],
                    help="study: closure outputs applied (flux,energy flux,ionization), one or more triples")
    ap.add_argument("--save", default=None, help="study: write the particle record and closures to this .npz")
    ap.add_argument("--load", default=None, help="study: take the particle record and closures from this .npz")
    a = ap.parse_args(argv)
    if a.what == "fluid":
        # a fluid screen of imposed fields 6..20 V/cm/Torr (neon, 1 Torr, L = 10 cm): time per step
        recs = transport()
        tab = Table(recs)
        states = [homogeneous_E0(tab, e, 1.0) for e in np.linspace(6.0, 20.0, a.columns)]
        r = fluid_screen(recs, states, L_m=0.10, n_cells=a.cells, steps=a.steps, diag_every=50)
        print(f"fluid: {a.columns} columns x {a.cells} cells, {a.steps} steps in {r['ms']:.2f} ms "
              f"({r['launches']} launches)", flush=True)
        return 0
    if a.what == "grid":
        # the particle model at 16 points of the (pR, I/R) screen against the fluid screen with the
        # closures of an earlier study (--load)
        r = grid_study(grid_points(), a.load, L_m=a.L, n_cells=a.pic_cells, fluid_cells=a.fluid_cells or 4096,
                       particles=a.particles, nu_bound=a.nu_bound, stencils=tuple(a.stencils), agg=a.agg,
                       train_steps=a.train_steps,
                       components=[[float(v) for v in c.split(",")] for c in a.components],
                       log=lambda s: print(s, flush=True))
        for k, (pr, ir) in enumerate(r["points"]):
            line = (f"pR={pr:.3g} I/R={ir:.3g}: E0={r['pic_E0'][k]:.4g} V/m PIC lam={r['pic'][k]['lam'] * 100:.3g} cm "
                    f"v={r['pic'][k]['v_ph']:.3g} g={r['pic'][k]['gamma']:.3g}")
            for name, obs in r["variants"].items():
                o = obs[k]
                line += f" | {name} lam={o['lam'] * 100:.3g}" if o else f" | {name} -"
            print(line, flush=True)
        if a.out:
            with open(a.out, "w") as fh:
                json.dump(_jsonable(r), fh, indent=1)
        return 0
    r = study([6, 8, 10, 12, 14, 16, 18, 20], [7, 9, 11, 13, 15, 17, 19, 21], L_m=a.L, n_cells=a.pic_cells,
              particles=a.particles, windows=a.windows, window=a.window, agg=a.agg, train_steps=a.train_steps,
              fluid_cells=a.fluid_cells, early=a.early, save=a.save, load=a.load,
              components=[[float(v) for v in c.split(",")] for c in a.components],
              nu_bound=a.nu_bound, stencils=tuple(a.stencils), log=lambda s: print(s, flush=True))
    for k, e in enumerate(r["E_compare"]):
        p, f, g, l, d = r["pic"][k], r["fluid"][k], r["fluid_closure"][k], r["linear"][k], r["dispersion"][k]
        print(f"E0/p={e}: PIC lam={p['lam'] * 100:.3g} cm v={p['v_ph']:.3g} m/s g={p['gamma']:.3g}/s | "
              f"fluid lam={f['lam'] * 100:.3g} v={f['v_ph']:.3g} g={f['gamma']:.3g} | fluid+closure "
              f"lam={g['lam'] * 100:.3g} v={g['v_ph']:.3g} | eq.22 lam={l['lam'] * 100:.3g} v={l['v_ph']:.3g} "
              f"g={l['gamma_max']:.3g} | full linear lam={d['lam'] * 100:.3g} g={d['gamma']:.3g}", flush=True)
    for c in r["closures"]:
        print(f"closure stencil {c['stencil']} components {c['components']}: held-out mse {c['mse_net']} "
              f"(table {c['mse_table']}); lambda cm "
              + " ".join(f"{x * 100:.3g}" for x in c["lam"]), flush=True)
    print("speed ratio (particle / fluid per column):",
          r["pic_seconds_per_column"] / r["fluid_seconds_per_column"], flush=True)
    if a.out:
        with open(a.out, "w") as fh:
            json.dump(_jsonable(r), fh, indent=1)
    return 0


if __name__ == "__main__":
    import sys
    sys.exit(main())
