"""Shared test helpers: parameter sets for the physics pins (inputs only)."""
import numpy as np

from paper_2202_03215_gb300 import workloads as w

QE = 1.602176634e-19
ME = 9.1093837015e-31
AMU = 1.66053906660e-27
KB = 1.380649e-23
EPS0 = 8.8541878128e-12
TORR = 133.32236842105263


def beam_state(n, n_cells, speed, rng, direction=(1.0, 0.0, 0.0), step=0, next_id=None,
               n_i=0, ion_speed=0.0, float32=False):
    """Mono-energetic electron beam (and optionally an ion beam) at random positions."""
    d = {}
    for sp, m, sv in (("e", n, speed), ("i", n_i, ion_speed)):
        cell = rng.integers(0, n_cells, m).astype(np.int32)
        off = rng.random(m)
        if float32:
            off = np.minimum(off.astype(np.float32), np.float32(0.99999994)).astype(np.float64)
        dvec = np.asarray(direction, dtype=np.float64)
        dvec = dvec / np.linalg.norm(dvec)
        v = np.outer(dvec, np.full(m, sv))
        if float32:
            v = v.astype(np.float32).astype(np.float64)
        d[f"cell_{sp}"], d[f"off_{sp}"] = cell, off
        d[f"vx_{sp}"], d[f"vy_{sp}"], d[f"vz_{sp}"] = v[0].copy(), v[1].copy(), v[2].copy()
    d["id_e"] = np.arange(n, dtype=np.uint64)
    d["id_i"] = np.arange(n, n + n_i, dtype=np.uint64)
    d["step"] = step
    d["next_id"] = n + n_i if next_id is None else next_id
    d["E0"] = 0.0
    d["E"] = None
    d["Q_i"] = None
    return d


def maxwell_model_xsec(nu, ng, eps_max, n_table):
    """sigma(eps) = nu / (n_g v(eps)) on the internal grid (constant collision frequency)."""
    de = eps_max / (n_table - 1)
    e = np.arange(n_table) * de
    v = np.sqrt(e * (2 * QE / ME))
    s = np.empty(n_table)
    s[1:] = nu / (ng * v[1:])
    s[0] = s[1]
    return w.XSec(w.ELASTIC, e, s)


def n_gas(p_torr=1.0, T=300.0):
    return p_torr * TORR / (KB * T)
