"""Seed ensembles of the particle model: the precision form against the FP64 form.

A run of the PIC-MCC column is a stochastic, chaotic trajectory: after a few
hundred steps the FP32 particle state of the precision form and the FP64 state
of the plain form have diverged at the rounding level, and so have two seeds of
one form.  What the two forms must share is the statistics of what the paper
reads off its runs (Sec. III, Fig. 4 and the x-t diagrams of Fig. 13): the
time-averaged moments, the striation wavelength and their phase velocity.  This
module runs `seeds` columns of each form as one GPU batch per form, samples the
moments every `diag_every` steps, averages them over the saturated part of the
record and compares the seed means of the two forms: the difference of the
means against three standard errors of that difference.

python -m paper_2202_03215_gb300.statistics [--seeds 8] [--out file.json]
"""
from __future__ import annotations

import argparse
import json
import math
from dataclasses import dataclass
from typing import Dict, List, Sequence

import numpy as np

from . import workloads as w

# outputs compared, with their units
OUTPUTS = {
    "mean_energy_eV": "eV",         # density-weighted column mean of the electron mean energy
    "electron_flux": "m^-2 s^-1",   # column mean of the electron flux (drift along the column)
    "ionization_rate": "m^-3 s^-1", # column mean of the ionization rate
    "density_modulation": "1",      # rms of n_e / <n_e> - 1 over the column: the striation amplitude
    "space_charge_field": "V/m",    # rms of E + E0 over the column: the striation field
    "lambda_cm": "cm",              # striation wavelength (mode of largest saturated power)
    "v_ph_mps": "m/s",              # phase velocity of that mode, positive toward the cathode
}


@dataclass
class Setup:
    E0_over_p: float = 14.0        # V/cm/Torr
    p_torr: float = 1.0
    L_m: float = 0.10
    n_cells: int = 2048
    particles: int = 1_000_000
    dt_s: float = 4e-11
    warm_steps: int = 60_000       # to the saturated state (growth rate ~4e6 /s at 14 V/cm/Torr)
    windows: int = 40
    window: int = 2000
    diag_every: int = 50
    n_modes: int = 64
    seed0: int = 101

    def params(self, seed: int, column: int, precision: int) -> w.Params:
        return w.config_neon_column(n_per_species=self.particles, precision=precision).with_(
            pressure_torr=self.p_torr, L_m=self.L_m, n_cells=self.n_cells, dt_s=self.dt_s,
            E0_Vpm=self.E0_over_p * 100.0 * self.p_torr, drive=w.DRIVE_E0, n0_m3=1e15,
            loss_mode=w.LOSS_PAIR, diag_every=self.diag_every, sort_every=1000, seed=seed, column=column)


def _column_outputs(m: dict, E0: float) -> Dict[str, float]:
    ne = m["n_e"]
    nbar = ne.mean()
    return {"mean_energy_eV": float((m["mean_eps_e"] * ne).sum() / max(ne.sum(), 1e-300)),
            "electron_flux": float(m["gamma_e"].mean()),
            "ionization_rate": float(m["iz_rate"].mean()),
            "density_modulation": float(np.sqrt(((ne / nbar - 1.0) ** 2).mean())) if nbar > 0 else math.nan,
            "space_charge_field": float(np.sqrt(((m["E"] + E0) ** 2).mean()))}


def run_form(setup: Setup, precision: int, seeds: int) -> List[Dict[str, float]]:
    """One batch of `seeds` columns of one storage form; per seed the time averages over the
    saturated windows and the striation observables of the whole record."""
    from . import Batch
    from .screen import observables
    params = [setup.params(setup.seed0 + k, k, precision) for k in range(seeds)]
    b = Batch(params)
    try:
        b.step(setup.warm_steps)
        for c in b.columns:
            c.moments(reset=True)
        M = setup.n_modes
        rec = np.zeros((setup.windows, seeds, M + 1), complex)
        acc = [[] for _ in range(seeds)]
        for s in range(setup.windows):
            b.step(setup.window)
            for k, c in enumerate(b.columns):
                m = c.moments(reset=True)
                F = np.fft.fft(m["n_e"]) / len(m["n_e"])
                rec[s, k, 0] = m["n_e"].mean()
                rec[s, k, 1:] = F[1:M + 1]
                acc[k].append(_column_outputs(m, params[k].E0_Vpm))
    finally:
        b.close()
    t = (np.arange(setup.windows) + 0.5) * setup.window * setup.dt_s
    out = []
    for k in range(seeds):
        d = {key: float(np.mean([a[key] for a in acc[k]])) for key in acc[k][0]}
        ob = observables(t, rec[:, k], setup.L_m)
        d["lambda_cm"] = 100.0 * ob["lam"]
        # the applied field points along -x: the cathode is at -x, waves toward it have v_ph < 0
        d["v_ph_mps"] = -ob["v_ph"]
        out.append(d)
    return out


def compare(a: Sequence[Dict[str, float]], b: Sequence[Dict[str, float]], resolution: Dict[str, float] | None = None):
    """Per output: seed means and standard deviations of both forms, the difference of the means,
    its standard error, and whether |difference| <= 3 standard errors.  `resolution` gives a
    floor for the standard error of a quantised output (the wavelength takes the values L/m)."""
    resolution = resolution or {}
    rows = {}
    for key in OUTPUTS:
        xa = np.array([r[key] for r in a], float)
        xb = np.array([r[key] for r in b], float)
        ma, mb = xa.mean(), xb.mean()
        sa = xa.std(ddof=1) if len(xa) > 1 else math.nan
        sb = xb.std(ddof=1) if len(xb) > 1 else math.nan
        se = math.sqrt(sa * sa / len(xa) + sb * sb / len(xb))
        se = max(se, resolution.get(key, 0.0))
        d = ma - mb
        rows[key] = {"mixed_mean": ma, "mixed_sd": sa, "fp64_mean": mb, "fp64_sd": sb, "diff": d,
                     "se_diff": se, "rel_diff": d / mb if mb else math.nan,
                     "band3": 3 * se, "within_3se": bool(abs(d) <= 3 * se), "unit": OUTPUTS[key]}
    return rows


def lambda_resolution(setup: Setup, lam_cm: float) -> float:
    """Step between adjacent wavelengths L/m and L/(m+1) near lam_cm, over sqrt(12): the
    standard deviation of the quantisation, a floor for the wavelength's standard error."""
    L = 100.0 * setup.L_m
    m = max(1.0, round(L / lam_cm))
    return (L / m - L / (m + 1)) / math.sqrt(12.0)


def study(setup: Setup, seeds: int) -> dict:
    import time
    t0 = time.perf_counter()
    mixed = run_form(setup, w.MIXED, seeds)
    t1 = time.perf_counter()
    fp64 = run_form(setup, w.FP64, seeds)
    t2 = time.perf_counter()
    lam = float(np.mean([r["lambda_cm"] for r in fp64]))
    rows = compare(mixed, fp64, {"lambda_cm": lambda_resolution(setup, lam) * math.sqrt(2.0 / seeds)})
    return {"setup": setup.__dict__, "seeds": seeds, "mixed": mixed, "fp64": fp64, "compare": rows,
            "seconds": {"mixed": t1 - t0, "fp64": t2 - t1}}


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--seeds", type=int, default=8)
    ap.add_argument("--particles", type=int, default=1_000_000)
    ap.add_argument("--E0-over-p", type=float, default=14.0)
    ap.add_argument("--warm", type=int, default=60_000)
    ap.add_argument("--windows", type=int, default=40)
    ap.add_argument("--window", type=int, default=2000)
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    s = Setup(E0_over_p=a.E0_over_p, particles=a.particles, warm_steps=a.warm, windows=a.windows, window=a.window)
    r = study(s, a.seeds)
    for k, v in r["compare"].items():
        print(f"{k:20s} mixed {v['mixed_mean']:.5g} +- {v['mixed_sd']:.2g}  fp64 {v['fp64_mean']:.5g} +- "
              f"{v['fp64_sd']:.2g}  diff {v['diff']:+.3g} ({v['rel_diff']:+.2%})  3se {v['band3']:.3g}  "
              f"{'ok' if v['within_3se'] else 'OUTSIDE'}")
    print("seconds", r["seconds"])
    if a.out:
        with open(a.out, "w") as f:
            json.dump(r, f, indent=1, default=float)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
