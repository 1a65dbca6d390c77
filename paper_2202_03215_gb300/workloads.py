"""Seeded synthetic inputs for the PIC-MCC positive-column workloads.

This module holds input generators only: gas constants, the analytic
cross-section shapes that stand in for the LXCat data the paper uses
(Sec. II: Phelps argon with one lumped excitation level, neon, ion-neutral
charge exchange), and the parameter sets of the five workloads.  It holds
none of the method's arithmetic.  Both the CUDA library and the CPU oracle
receive the same tables from here as plain arrays.

Cross-section readings (the paper gives only database names, so the shapes
are synthetic):
  argon  elastic    6e-20*exp(-e/0.05) + 1.5e-19*exp(-ln(e/12)^2/2), floor 1e-22 m^2
                    (peak 1.5e-19 m^2 near 12 eV, Ramsauer minimum ~3e-22 near 0.3 eV)
         excitation Lotz form, threshold 11.5 eV, peak 2e-21 m^2
         ionization Lotz form, threshold 15.76 eV, peak 3e-20 m^2
         ion CX     5e-19 m^2 constant
  neon   elastic    2e-20 m^2 flat
         excitation Lotz form, threshold 16.6 eV, peak 4e-21 m^2
         ionization Lotz form, threshold 21.56 eV, peak 7e-21 m^2
         ion CX     3e-19 m^2 constant
Lotz form: sigma = s_pk * e * ln(u) / u, u = eps/threshold (peak s_pk at u = e).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import List, Optional

import numpy as np

# process kinds (same numbering in include/pic.h and the oracle's header)
ELASTIC, EXCITATION, IONIZATION, ION_CX, ION_ISO = 0, 1, 2, 3, 4
# drive modes
DRIVE_E0, DRIVE_V, DRIVE_CIRCUIT, DRIVE_RI = 0, 1, 2, 3
# field modes
FIELD_POISSON, FIELD_APPLIED = 0, 1
# loss modes
LOSS_PAIR, LOSS_RADIAL, LOSS_NONE, LOSS_SWARM = 0, 1, 2, 3
FLAG_RECORD_CODES, FLAG_NO_GRAPH, FLAG_ALLOW_LARGE_NULL, FLAG_BOUNDED = 1, 2, 4, 8
# particle storage forms
FP64, MIXED = 0, 1

AMU_AR = 39.948
AMU_NE = 20.1797


@dataclass
class XSec:
    kind: int
    energy_eV: np.ndarray
    sigma_m2: np.ndarray
    threshold_eV: float = 0.0


def _energy_grid(eps_max: float, n: int = 1200, threshold: float = 0.0) -> np.ndarray:
    g = np.concatenate([[0.0], np.geomspace(1e-3, eps_max, n - 1)])
    if threshold > 0.0:
        g = np.unique(np.concatenate([g, [threshold]]))
    return g


def _lotz(eps: np.ndarray, thr: float, peak: float) -> np.ndarray:
    u = np.maximum(eps / thr, 1.0)
    s = peak * math.e * np.log(u) / u
    s[eps < thr] = 0.0
    return s


def argon_xsecs(eps_max_e: float = 500.0, eps_max_i: float = 50.0,
                sigma_iso: float = 0.0) -> List[XSec]:
    g = _energy_grid(eps_max_e)
    with np.errstate(divide="ignore"):
        ln = np.where(g > 0, np.log(np.where(g > 0, g, 1.0) / 12.0), -np.inf)
    el = 6e-20 * np.exp(-g / 0.05) + 1.5e-19 * np.exp(-0.5 * ln * ln)
    el = np.maximum(el, 1e-22)
    gx = _energy_grid(eps_max_e, threshold=11.5)
    gi = _energy_grid(eps_max_e, threshold=15.76)
    out = [XSec(ELASTIC, g, el),
           XSec(EXCITATION, gx, _lotz(gx, 11.5, 2e-21), 11.5),
           XSec(IONIZATION, gi, _lotz(gi, 15.76, 3e-20), 15.76)]
    ge = np.array([0.0, eps_max_i])
    out.append(XSec(ION_CX, ge, np.array([5e-19, 5e-19])))
    if sigma_iso > 0.0:
        out.append(XSec(ION_ISO, ge, np.array([sigma_iso, sigma_iso])))
    return out


def neon_xsecs(eps_max_e: float = 200.0, eps_max_i: float = 50.0,
               sigma_iso: float = 0.0) -> List[XSec]:
    g = _energy_grid(eps_max_e)
    gx = _energy_grid(eps_max_e, threshold=16.6)
    gi = _energy_grid(eps_max_e, threshold=21.56)
    out = [XSec(ELASTIC, g, np.full_like(g, 2e-20)),
           XSec(EXCITATION, gx, _lotz(gx, 16.6, 4e-21), 16.6),
           XSec(IONIZATION, gi, _lotz(gi, 21.56, 7e-21), 21.56)]
    ge = np.array([0.0, eps_max_i])
    out.append(XSec(ION_CX, ge, np.array([3e-19, 3e-19])))
    if sigma_iso > 0.0:
        out.append(XSec(ION_ISO, ge, np.array([sigma_iso, sigma_iso])))
    return out


def neon_multilevel_xsecs(eps_max_e: float = 200.0, eps_max_i: float = 50.0) -> List[XSec]:
    """Synthetic neon with the excitation split over seven levels (the lumped level of
    neon_xsecs spread over thresholds 16.6 .. 20.0 eV, Lotz forms whose peaks sum to its 4e-21 m^2),
    for the multi-level machinery; elastic, ionization and charge exchange as in neon_xsecs."""
    g = _energy_grid(eps_max_e)
    gi = _energy_grid(eps_max_e, threshold=21.56)
    out = [XSec(ELASTIC, g, np.full_like(g, 2e-20))]
    thr = [16.6, 16.7, 16.85, 18.4, 18.7, 19.0, 20.0]
    peak = [1.0e-21, 0.5e-21, 0.5e-21, 0.8e-21, 0.5e-21, 0.4e-21, 0.3e-21]
    for t, s in zip(thr, peak):
        gx = _energy_grid(eps_max_e, threshold=t)
        out.append(XSec(EXCITATION, gx, _lotz(gx, t, s), t))
    out.append(XSec(IONIZATION, gi, _lotz(gi, 21.56, 7e-21), 21.56))
    ge = np.array([0.0, eps_max_i])
    out.append(XSec(ION_CX, ge, np.array([3e-19, 3e-19])))
    return out


@dataclass
class Params:
    """Problem statement of one periodic positive column (Sec. II)."""
    gas_mass_amu: float = AMU_AR
    pressure_torr: float = 1.0
    T_gas_K: float = 300.0
    L_m: float = 0.05
    R_m: float = 0.01
    drive: int = DRIVE_V
    field_mode: int = FIELD_POISSON
    E0_Vpm: float = 0.0
    V_applied: float = 20.0
    I_A: float = 0.0
    U_src: float = 0.0
    R_ext_ohm_m2: float = 0.0
    xsec: List[XSec] = field(default_factory=argon_xsecs)
    n_cells: int = 500
    ion_subcycle: int = 10
    dt_s: float = 2e-11
    n_e0: int = 100_000
    n_i0: int = 100_000
    capacity: int = 0
    n0_m3: float = 1e15
    Te0_eV: float = 2.0
    Ti0_eV: float = 0.026
    loss_mode: int = LOSS_PAIR
    precision: int = FP64
    nu_w: float = 0.0
    seed: int = 1
    diag_every: int = 0
    sort_every: int = 0
    n_table: int = 8193
    flags: int = 0
    eps_max_e_eV: float = 500.0
    eps_max_i_eV: float = 50.0
    column: int = 0
    J_emit_Am2: float = 0.0       # bounded column (FLAG_BOUNDED): cathode emission current density
    T_emit_eV: float = 0.0        # and its emission temperature

    @property
    def n_nodes(self) -> int:
        """Entries of the node arrays: n_cells, or n_cells + 1 between two electrodes."""
        return self.n_cells + (1 if self.flags & FLAG_BOUNDED else 0)

    def with_(self, **kw) -> "Params":
        return replace(self, **kw)


def config_argon_small(seed: int = 1, **kw) -> Params:
    """Argon 1 Torr 300 K, L = 5 cm, 500 cells, dt = 2e-11 s, ions subcycled x10,
    1e5 electrons + 1e5 ions, n0 = 1e15 m^-3, Te0 = 2 eV, Ti0 = 0.026 eV,
    20 V applied (E0 = 400 V/m), PAIR loss, FP64 particle storage."""
    p = Params(seed=seed)
    return p.with_(**kw) if kw else p


def config_neon_column(seed: int = 1, precision: int = MIXED, n_per_species: int = 20_000_000,
                       E0_Vpm: float = 600.0, **kw) -> Params:
    """Neon 1 Torr 300 K, L = 30 cm, R = 1 cm, 16384 cells, 2e7 particles per species,
    dt = 4e-11 s, ions subcycled x10, int32 cell + FP32 offset/velocity storage, sorted by cell
    every 100 steps (the fastest whole step measured: 0.250 ms, against 0.255 ms at 250 and
    0.268 ms at 50)."""
    p = Params(gas_mass_amu=AMU_NE, L_m=0.30, R_m=0.01, drive=DRIVE_E0, E0_Vpm=E0_Vpm,
               V_applied=0.0, xsec=neon_xsecs(), n_cells=16384, dt_s=4e-11,
               n_e0=n_per_species, n_i0=n_per_species, precision=precision, seed=seed,
               eps_max_e_eV=200.0, sort_every=100, diag_every=0)
    return p.with_(**kw) if kw else p


def random_state(n: int, n_cells: int, rng: np.random.Generator, v_scale: float,
                 float32: bool = False, id0: int = 0):
    """A seeded synthetic particle state: cells, offsets in [0,1), Gaussian velocities.
    float32=True makes every value exactly representable in FP32."""
    cell = rng.integers(0, n_cells, size=n, dtype=np.int32)
    off = rng.random(n)
    v = rng.standard_normal((3, n)) * v_scale
    if float32:
        off = off.astype(np.float32).astype(np.float64)
        off[off >= 1.0] = np.nextafter(np.float32(1.0), np.float32(0.0))
        v = v.astype(np.float32).astype(np.float64)
    ids = np.arange(id0, id0 + n, dtype=np.uint64)
    return cell, off, v[0].copy(), v[1].copy(), v[2].copy(), ids


def config_batch_sweep(n_columns: int = 64, seed: int = 42, particle_scale: float = 1.0,
                       precision: int = MIXED) -> List[Params]:
    """Batched sweep of uneven columns: log-uniform draws from `seed` of
    L in [0.05, 0.40] m, p in [0.3, 3] Torr, I in [0.1, 5] mA and 1e5..5e6 particles
    per species; cells = round(L / 0.05 m * 2048) clamped to [2048, 16384]; gases
    alternate argon / neon.  Readings (no drive from current is built): E0/p = 12 V/cm/Torr
    for argon and 6 V/cm/Torr for neon (near the paper's striation onsets); n0 = 1e15 m^-3
    x (I / 1 mA) (the model is linear in density); dt = 5e-12 s for every column (the
    batch shares one time step; nu* dt <= 0.3 up to 3 Torr with 200 eV tables)."""
    rng = np.random.default_rng(seed)

    def logu(a, b):
        return float(np.exp(rng.uniform(np.log(a), np.log(b))))

    out = []
    for c in range(n_columns):
        L, p, I, n = logu(0.05, 0.40), logu(0.3, 3.0), logu(1e-4, 5e-3), logu(1e5, 5e6)
        n = max(1000, int(n * particle_scale))
        cells = int(min(16384, max(2048, round(L / 0.05 * 2048))))
        argon = c % 2 == 0
        xs = argon_xsecs(eps_max_e=200.0) if argon else neon_xsecs()
        out.append(Params(gas_mass_amu=AMU_AR if argon else AMU_NE, pressure_torr=p, L_m=L, R_m=0.01,
                          drive=DRIVE_E0, E0_Vpm=(1200.0 if argon else 600.0) * p, V_applied=0.0, I_A=I,
                          xsec=xs, n_cells=cells, dt_s=5e-12, ion_subcycle=10, n_e0=n, n_i0=n,
                          n0_m3=1e15 * (I / 1e-3), precision=precision, seed=seed, sort_every=1000,
                          eps_max_e_eV=200.0, column=c))
    return out
