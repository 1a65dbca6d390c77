"""Two-term Boltzmann solve of a uniform-field electron swarm (oracle side).

TEST INFRASTRUCTURE ONLY: used by tests/ to pin the particle swarms and the
library's own transport tables; the product path never imports it.

The paper obtains the fluid-model closure (Sec. IV.A, eqs. 6-9: nu_i, L_eps,
mu_e, D_e, mu_eps, D_eps as functions of the electron temperature) from
steady-state homogeneous solutions of the two-term Boltzmann equation, and
states that uniform-field PIC-MCC reproduces them (Sec. III.B).  This module
writes that equation out directly, in plain FP64:

  EEDF F(eps), normalised so that int eps^(1/2) F deps = 1; all rates per gas
  density N; gamma = (2e/m)^(1/2).  Steady state, no spatial gradient:

    d/deps G(eps) = S(eps)
    G = -(gamma/3) (E/N)^2 (eps/sigma_m) dF/deps - gamma (2m/M) eps^2 sigma_el F

  G is the upward flux in energy (field heating minus elastic cooling; the
  neutrals are at rest for electrons, as in the particle model), sigma_m the
  momentum-transfer cross section (every process scatters isotropically, so
  it is the sum of all electron cross sections) and S the inelastic
  redistribution: an excitation moves electrons from eps to eps - u_k; an
  ionization leaves the scattered electron uniformly on [0, eps - u_iz] and
  creates no new electron (the particle model's swarm mode, in which the
  population is held fixed and ionizations are only counted).

Discretisation (plain finite volumes, chosen to be different from the
library's exponential scheme): cell centres eps_i = (i + 1/2) d, central
differences for the face fluxes, zero flux at both ends, redistributed
electrons deposited conservatively (linear weights for a shift, exact
overlaps for the uniform interval), one row replaced by the normalisation,
dense solve.

Transport integrals (per N):
  mu N     = -(gamma/3)        int eps/sigma_m dF/deps deps
  D N      =  (gamma/3)        int eps/sigma_m F deps
  mu_eps N = -(gamma/(3 ebar)) int eps^2/sigma_m dF/deps deps
  D_eps N  =  (gamma/(3 ebar)) int eps^2/sigma_m F deps
  nu_k / N =   gamma           int eps sigma_k F deps
"""
from __future__ import annotations

import numpy as np

QE = 1.602176634e-19
ME = 9.1093837015e-31
AMU = 1.66053906660e-27
GAMMA = np.sqrt(2.0 * QE / ME)
TD = 1e-21

ELASTIC, EXCITATION, IONIZATION = 0, 1, 2


def sigma_at(xs, eps):
    """Cross section (kind, threshold, energy[], sigma[]) at eps: linear
    interpolation, last value held above the table, zero below a threshold."""
    kind, thr, e, s = xs
    out = np.interp(eps, np.asarray(e, float), np.asarray(s, float))
    if kind != ELASTIC:
        out = np.where(eps < thr, 0.0, out)
    return out


def solve(xsecs, mass_amu, EN_Td, eps_max=100.0, n=2000):
    """Two-term EEDF and transport at reduced field EN_Td.

    xsecs: electron processes as (kind, threshold_eV, energy_eV[], sigma_m2[]).
    Returns a dict with the grid, F and the swarm quantities (SI, per N where
    noted)."""
    d = eps_max / n
    ec = (np.arange(n) + 0.5) * d           # cell centres
    ef = np.arange(1, n) * d                # interior faces
    EN = EN_Td * TD
    mratio = 2.0 * ME / (mass_amu * AMU)
    sig_c = [sigma_at(x, ec) for x in xsecs]
    sig_f = [sigma_at(x, ef) for x in xsecs]
    sm_c = np.sum(sig_c, axis=0)
    sm_f = np.sum(sig_f, axis=0)
    sel_f = np.sum([s for x, s in zip(xsecs, sig_f) if x[0] == ELASTIC], axis=0)

    A = (GAMMA / 3.0) * EN * EN * ef / sm_f           # field diffusion coefficient at faces
    B = GAMMA * mratio * ef * ef * sel_f              # elastic cooling drift at faces
    peclet = B * d / A
    if np.max(peclet) >= 2.0:
        raise ValueError("grid too coarse for central differences (cell Peclet %.2f)" % np.max(peclet))

    M = np.zeros((n, n))
    # flux through face i+1/2: G = F_i (A/d - B/2) + F_{i+1} (-A/d - B/2)
    gi = A / d - B / 2.0
    gj = -A / d - B / 2.0
    i = np.arange(n - 1)
    M[i, i] += gi            # + G_{i+1/2} in row i
    M[i, i + 1] += gj
    M[i + 1, i] -= gi        # - G_{i+1/2} in row i+1
    M[i + 1, i + 1] -= gj

    lo = np.arange(n) * d    # cell lower edges
    for x, s in zip(xsecs, sig_c):
        kind, thr = x[0], x[1]
        if kind == ELASTIC:
            continue
        R = d * GAMMA * ec * s                       # loss rate out of cell j per unit F_j
        M[np.arange(n), np.arange(n)] += R
        for j in np.nonzero(s > 0.0)[0]:
            top = ec[j] - thr                        # energy left after the threshold
            if top < 0.0:
                continue
            if kind == EXCITATION:
                pos = top / d - 0.5                  # in cell-centre index units
                k = int(np.floor(pos))
                if k < 0:
                    M[0, j] -= R[j]
                else:
                    fr = pos - k
                    M[k, j] -= R[j] * (1.0 - fr)
                    M[min(k + 1, n - 1), j] -= R[j] * fr
            else:
                if top == 0.0:
                    M[0, j] -= R[j]
                    continue
                ov = np.clip(np.minimum(lo + d, top) - lo, 0.0, None) / top
                M[:, j] -= R[j] * ov
    M[n - 1, :] = np.sqrt(ec) * d
    rhs = np.zeros(n)
    rhs[n - 1] = 1.0
    scale = 1.0 / np.max(np.abs(M), axis=1)          # row equilibration before the dense solve
    F = np.linalg.solve(M * scale[:, None], rhs * scale)

    dF = np.diff(F)                                  # F_{i+1} - F_i at interior faces
    ebar = np.sum(ec ** 1.5 * F) * d
    muN = -(GAMMA / 3.0) * np.sum(ef / sm_f * dF)
    DN = (GAMMA / 3.0) * np.sum(ec / sm_c * F) * d
    mueN = -(GAMMA / (3.0 * ebar)) * np.sum(ef * ef / sm_f * dF)
    DeN = (GAMMA / (3.0 * ebar)) * np.sum(ec * ec / sm_c * F) * d
    nuN = [GAMMA * np.sum(ec * s * F) * d for s in sig_c]
    sel_c = np.sum([s for x, s in zip(xsecs, sig_c) if x[0] == ELASTIC], axis=0)
    loss_el = GAMMA * mratio * np.sum(ec * ec * sel_c * F) * d
    loss_inel = 0.0
    loss_swarm_iz = 0.0
    nu_iz = 0.0
    for x, s, nu in zip(xsecs, sig_c, nuN):
        if x[0] == EXCITATION:
            loss_inel += x[1] * nu
        elif x[0] == IONIZATION:
            loss_inel += x[1] * nu
            nu_iz += nu
            # swarm mode: the scattered electron keeps on average half of eps - u_iz
            loss_swarm_iz += GAMMA * np.sum(ec * s * F * (0.5 * (ec + x[1]) - x[1])) * d
    w = muN * EN
    return dict(eps=ec, F=F, mean_eps=ebar, Te=2.0 / 3.0 * ebar, muN=muN, DN=DN, mueN=mueN, DeN=DeN,
                nuN=nuN, nu_izN=nu_iz, drift=w, alphaN=nu_iz / w if w > 0 else 0.0,
                loss_elN=loss_el, loss_N=loss_el + loss_inel,
                power_N=muN * EN * EN, swarm_loss_N=loss_el + loss_inel + loss_swarm_iz)


KB = 1.380649e-23
TORR = 133.32236842105263
ION_CX, ION_ISO = 3, 4
J0_ZERO = 2.405            # first zero of J_0: the "2.4" of eq. 2


def ion_mobility_N(ion_xsecs, mass_amu, T_K):
    """mu_i N of ions in their parent gas at low field, the ion mobility of eq. 2 (the
    paper takes measured values; the synthetic gases here have a cross section only).
    First Chapman-Enskog approximation for a constant momentum-transfer cross section Q:
    mu_i = 3 e / (16 N Q) (2 pi / (m_r k T))^(1/2), m_r = M/2 for an ion in its own gas.
    Q is read at the mean relative energy of a thermal pair, 8 k T / pi: a charge
    exchange reverses the ion's velocity in the centre-of-mass frame (2 sigma_cx), an
    isotropic collision transfers sigma_iso on average."""
    eps = 8.0 * KB * T_K / (np.pi * QE)
    Q = 0.0
    for kind, thr, e, s in ion_xsecs:
        if kind == ION_CX:
            Q += 2.0 * float(np.interp(eps, np.asarray(e, float), np.asarray(s, float)))
        elif kind == ION_ISO:
            Q += float(np.interp(eps, np.asarray(e, float), np.asarray(s, float)))
    return 3.0 * QE / (16.0 * Q) * np.sqrt(2.0 * np.pi / (0.5 * mass_amu * AMU * KB * T_K))


def ri_drive(xsecs, mass_amu, p_torr, T_K, R_m, I_A, eps_max, n=800, iters=40):
    """Field and density of a column of radius R carrying the current I (Sec. II, eq. 2).

    Ionization balances ambipolar loss to the wall, nu_i = (2.405/R)^2 D_a with
    D_a = D_e mu_i / mu_e, all at the homogeneous field E0; the electron terms come from
    this module's two-term solve at E0/N, mu_i from ion_mobility_N.  The balance
    N nu_izN - mu_i (D N / mu N) (2.405/R)^2 rises with E/N through zero; bisection on
    log(E/N) over [5, 300] Td (the central differences need some field at the grid's
    resolution; columns of the paper's range sit well inside).  The density follows from J = I / (pi R^2) =
    e n0 (mu_e + mu_i) E0.  Returns (E0 in V/m, n0 in m^-3, mu_i N)."""
    N = p_torr * TORR / (KB * T_K)
    el = [x for x in xsecs if x[0] in (ELASTIC, EXCITATION, IONIZATION)]
    ions = [x for x in xsecs if x[0] in (ION_CX, ION_ISO)]
    mu_i = ion_mobility_N(ions, mass_amu, T_K) / N
    g2 = (J0_ZERO / R_m) ** 2

    def balance(EN):
        s = solve(el, mass_amu, EN, eps_max=eps_max, n=n)
        return N * s["nu_izN"] - mu_i * (s["DN"] / s["muN"]) * g2, s

    lo, hi = np.log(5.0), np.log(300.0)
    if not (balance(np.exp(lo))[0] < 0.0 < balance(np.exp(hi))[0]):
        raise ValueError("no root of eq. 2 in [5, 300] Td")
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if balance(np.exp(mid))[0] < 0.0:
            lo = mid
        else:
            hi = mid
    EN = np.exp(0.5 * (lo + hi))
    _, s = balance(EN)
    E0 = EN * TD * N
    J = I_A / (np.pi * R_m ** 2)
    n0 = J / (QE * (s["muN"] / N + mu_i) * E0)
    return E0, n0, mu_i * N
