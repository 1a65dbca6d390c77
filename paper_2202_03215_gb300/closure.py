"""Data for the learned closure of the three-moment quasi-neutral fluid model
(Sec. IV.A, eqs. 3-9), produced by the GPU PIC-MCC library.

Two sources, both run through the C ABI on the GPU:
  * uniform-field electron swarms (field = applied only, ionizations counted
    but no particle created, Sec. III.B's "uniform field PIC"): transport
    versus reduced field E/N -- drift velocity, mean energy, ionization and
    energy-loss frequencies; these also give the tabulated closure of the
    fluid model (the paper's BOLSIG+ tables);
  * self-consistent columns: time-averaged moment windows (pic_moments) of
    the particle step, from which every interior cell gives one sample.

A sample maps the 5-point stencil of (n_e / <n_e>, mean energy, E / N) around
a cell to the electron flux per electron Gamma_e / n_e, the energy flux per
electron H_e / n_e and the ionization frequency nu_iz = (ionization rate) / n_e
at that cell (the model is linear in density, Sec. II, so per-electron targets
carry no density scale).  Features and targets are then normalised by fixed
scales (FEATURE_SCALE, TARGET_SCALE).
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Sequence

import numpy as np

from . import Batch
from . import workloads as w

TD = 1e-21            # 1 Townsend in V m^2
KB = 1.380649e-23

# normalisation of the 15 features (n / <n> x5, mean energy [eV] x5, E/N [Td] x5)
FEATURE_SCALE = np.array([1.0] * 5 + [10.0] * 5 + [50.0] * 5, dtype=np.float32)
# normalisation of the 3 targets (Gamma/n [m/s], H/n [eV m/s], nu_iz [1/s])
TARGET_SCALE = np.array([1e5, 1e6, 1e7], dtype=np.float32)


@dataclass
class SwarmPoint:
    EN_Td: float
    mean_eps_eV: float
    drift_mps: float          # electron drift velocity along -E (positive)
    nu_iz: float              # ionizations per electron per second
    loss_eVps: float          # energy loss per electron per second (= power gained in steady state)
    Te_eV: float


def n_gas(p: w.Params) -> float:
    return p.pressure_torr * 133.32236842105263 / (KB * p.T_gas_K)


def swarm_params(EN_Td: float, gas: str = "neon", n: int = 100_000, n_cells: int = 128, seed: int = 3,
                 column: int = 0) -> w.Params:
    """A uniform-field electron swarm in the periodic column (no space charge, ionizations counted)."""
    base = w.config_neon_column(n_per_species=n) if gas == "neon" else w.config_argon_small(n_e0=n)
    p = base.with_(n_cells=n_cells, L_m=0.01, field_mode=w.FIELD_APPLIED, drive=w.DRIVE_E0,
                   loss_mode=w.LOSS_SWARM, n_i0=0, ion_subcycle=0, sort_every=0, precision=w.MIXED,
                   dt_s=1e-11, seed=seed, column=column, diag_every=20, Te0_eV=3.0, flags=4)
    N = n_gas(p)
    return p.with_(E0_Vpm=EN_Td * TD * N)


def run_windows(params: Sequence[w.Params], warmup: int, windows: int, window: int):
    """Advance the columns as one GPU batch; return, per column, its moment windows and
    the ionization events counted over all windows."""
    b = Batch(params)
    if warmup:
        b.step(warmup)
    for c in b.columns:
        c.moments(reset=True)
    births0 = [c.stats()["births"] for c in b.columns]
    out = [[] for _ in params]
    for _ in range(windows):
        b.step(window)
        for k, c in enumerate(b.columns):
            out[k].append(c.moments(reset=True))
    births = [c.stats()["births"] - b0 for c, b0 in zip(b.columns, births0)]
    b.close()
    return out, births


def swarm_table(EN_Td: Sequence[float], gas: str = "neon", n: int = 100_000, relax: int = 3000,
                windows: int = 4, window: int = 500):
    """Uniform-field swarms at the given reduced fields (one GPU batch).  Returns the
    transport table and the per-window moments (sample sources)."""
    ps = [swarm_params(e, gas, n=n, column=i) for i, e in enumerate(EN_Td)]
    mom, births = run_windows(ps, relax, windows, window)
    table = []
    for e, p, ms, nb in zip(EN_Td, ps, mom, births):
        ne = sum(m["n_e"].sum() for m in ms)
        gam = sum(m["gamma_e"].sum() for m in ms)
        eps = sum((m["mean_eps_e"] * m["n_e"]).sum() for m in ms) / ne
        wdrift = gam / ne
        nu = nb / (p.n_e0 * windows * window * p.dt_s)
        table.append(SwarmPoint(e, eps, wdrift, nu, p.E0_Vpm * wdrift, 2.0 / 3.0 * eps))
    return table, ps, mom


def _stencil(a: np.ndarray, j: np.ndarray, step: int = 1) -> np.ndarray:
    N = len(a)
    return np.stack([a[(j + d * step) % N] for d in (-2, -1, 0, 1, 2)], 1)


def samples_from_moments(m: dict, p: w.Params) -> tuple[np.ndarray, np.ndarray]:
    """(features, targets) of every cell of one moment window of a periodic column."""
    N = len(m["n_e"])
    ng = n_gas(p)
    ne = np.maximum(m["n_e"], 1e-30)
    nbar = ne.mean()
    j = np.arange(N)
    X = np.concatenate([_stencil(ne / nbar, j), _stencil(m["mean_eps_e"], j),
                        _stencil(-m["E"] / (ng * TD), j)], 1)   # E/N along the drift direction
    T = np.stack([m["gamma_e"] / ne, m["heat_e"] / ne, m["iz_rate"] / ne], 1)
    return X.astype(np.float32), T.astype(np.float32)


def column_samples(params: Sequence[w.Params], steps: int, window: int, warmup: int = 0):
    """Moment-window samples of self-consistent columns advanced as one batch."""
    mom, _ = run_windows(params, warmup, max(1, steps // window), window)
    Xs, Ts = [], []
    for p, ms in zip(params, mom):
        for m in ms:
            X, T = samples_from_moments(m, p)
            Xs.append(X)
            Ts.append(T)
    return np.concatenate(Xs), np.concatenate(Ts)


def swarm_samples(ps: Sequence[w.Params], mom) -> tuple[np.ndarray, np.ndarray]:
    """Uniform-field samples: every cell of every swarm window."""
    Xs, Ts = [], []
    for p, ms in zip(ps, mom):
        for m in ms:
            X, T = samples_from_moments(m, p)
            Xs.append(X)
            Ts.append(T)
    return np.concatenate(Xs), np.concatenate(Ts)


def normalise(X: np.ndarray, T: np.ndarray):
    return X / FEATURE_SCALE, T / TARGET_SCALE


# ---------------------------------------------------------------------------
# Residual targets for the fluid screen: the network learns what the particle
# model's moments add to the tabulated closure of the fluid model, in the
# fluid model's frame (applied field along +x; the particle model's points
# along -x, so its windows are mirrored first).

def mirror(m: dict) -> dict:
    """x -> -x of a periodic moment window: node j -> node (-j) mod N; fluxes and the
    field change sign."""
    out = {}
    for k, v in m.items():
        if not isinstance(v, np.ndarray):
            out[k] = v
            continue
        r = np.roll(v[::-1], 1)
        out[k] = -r if k in ("gamma_e", "heat_e", "gamma_i", "E") else r
    return out


def _face(v):
    return 0.5 * (v + np.roll(v, -1))


def table_closure(n, T, Gamma_T, L_m, N_gas, mu_iN, tab):
    """The fluid model's tabulated closure evaluated on a given state (the same
    formulas as the fluid step): electron flux (eq. 11), field (eqs. 10 + 12) and energy
    flux (eqs. 8-9) at cells as averages of their faces, and nu_i(T)."""
    dx = L_m / len(n)
    mu_e = tab.at("muN", T) / N_gas
    D_e = tab.at("DN", T) / N_gas
    mu_eps = tab.at("mueN", T) / N_gas
    D_eps = tab.at("DeN", T) / N_gas
    mu_i = mu_iN / N_gas
    a = mu_i / (mu_e + mu_i)
    af = _face(a)
    nD = n * D_e
    G = -af * (np.roll(nD, -1) - nD) / dx - (1.0 - af) * Gamma_T
    nf = _face(n)
    E = -(np.roll(nD, -1) - nD) / (dx * nf * _face(mu_e)) + Gamma_T / (nf * _face(mu_e + mu_i))
    nT = n * T
    H = -0.75 * _face(mu_eps) * E * (nT + np.roll(nT, -1)) - 1.5 * (np.roll(n * D_eps * T, -1) - n * D_eps * T) / dx
    cell = lambda f: 0.5 * (f + np.roll(f, 1))
    return cell(G), cell(H), tab.at("nu_izN", T) * N_gas, cell(E)


def residual_samples(m: dict, p: w.Params, tab, mu_iN: float, T_range=None, step: int = 1):
    """(features, residual targets) of every cell of one particle-model window, in the
    fluid frame: features as the fluid screen computes them at stencil spacing `step`
    (n/<n>, mean energy, E/N
    from eq. 17), targets = (Gamma_e - Gamma_tab)/n, (H_e - H_tab)/n, nu_iz - nu_tab."""
    f = mirror(m)
    N_gas = n_gas(p)
    n = np.maximum(f["n_e"], 1e-30 + 1e-6 * f["n_e"].mean())
    T = 2.0 / 3.0 * f["mean_eps_e"]
    if T_range is not None:
        T = np.clip(T, *T_range)
    Gamma_T = float(np.mean(f["gamma_i"] - f["gamma_e"]))
    G, H, nu, E = table_closure(n, T, Gamma_T, p.L_m, N_gas, mu_iN, tab)
    j = np.arange(len(n))
    X = np.concatenate([_stencil(n / n.mean(), j, step), _stencil(1.5 * T, j, step),
                        _stencil(E / (N_gas * TD), j, step)], 1)
    Y = np.stack([(f["gamma_e"] - G) / n, (f["heat_e"] - H) / n, f["iz_rate"] / n - nu], 1)
    return X.astype(np.float32), Y.astype(np.float32)
