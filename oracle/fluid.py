"""Quasi-neutral three-moment fluid model of the positive column (oracle side).

TEST INFRASTRUCTURE ONLY: used by tests/ to check the library's fluid screen;
the product path never imports it.  Plain FP64 numpy, one column at a time,
the cyclic tridiagonal systems solved by a sparse direct solve.

Model (Sec. IV.A): electron continuity and energy, eqs. (3)-(4),
    d_t n + d_x Gamma = n (nu_i - nu_w)
    d_t (3/2 n T) + d_x H = P - n L_eps,       P = -Gamma E       (eq. 5)
with the flux of eq. (11) (eq. 7 with E eliminated through eq. 10)
    Gamma = -mu_i/(mu_e + mu_i) d_x(n D_e) - mu_e/(mu_e + mu_i) Gamma_T,
the field of eq. (10) combined with the flux of eq. (12), which is how eq. (17)
is obtained (read with mu_e outside the gradient, as that combination gives;
the printed eq. 17 moves it inside, which with a Te-dependent mobility adds a
negative effective heat conduction and makes the model ill-posed at high Te)
    E = -d_x(n D_e)/(n mu_e) + Gamma_T / (n (mu_e + mu_i)),
and the energy flux of eq. (8), H = -n beta E - d_x(n G), with eq. (9) read
as beta = 3/2 T mu_eps, G = 3/2 T D_eps (the form eq. 16's second line
requires).  mu_e, D_e, mu_eps, D_eps, nu_i and L_eps are functions of T
tabulated from uniform-field two-term solutions (eqs. 6-9), mu_i is constant,
Gamma_T = J/e is the constant total particle flux.

Discretisation (periodic, N cells, dx = L/N, faces j+1/2 between j and j+1;
face values of a, b, mu_eps, mu_e + mu_i and n are averages of the two
cells; coefficients from the table at the step's starting T):
 1. continuity, backward Euler in the diffusion and the losses, explicit in the
    rest (ionization explicit, losses implicit: n' stays positive):
      n'_j (1 + dt nu_w) - dt/dx^2 [a_{j+1/2} ((nD)'_{j+1} - (nD)'_j) - a_{j-1/2} ((nD)'_j - (nD)'_{j-1})]
          + dt/dx (dG_{j+1/2} - dG_{j-1/2})
        = n_j + dt/dx (b_{j+1/2} - b_{j-1/2}) Gamma_T + dt n_j (nu_i,j + dnu_j)
    a = mu_i/(mu_e + mu_i), b = mu_e/(mu_e + mu_i) at cells, D = D_e;
 2. Gamma_{j+1/2} from n' (eq. 11) plus dG_{j+1/2}; E_{j+1/2} from n' (eq. 17);
 3. energy, backward Euler in T' for the conduction, the energy drift and the
    linearised loss L(T') ~ L(T) + L'(T)(T' - T):
      3/2 (n'_j T'_j - n_j T_j)/dt + (H_{j+1/2} - H_{j-1/2})/dx
        = P_j - n'_j (L_j + L'_j (T'_j - T_j)),
      H_{j+1/2} = -3/4 mu_eps E (n'_j T'_j + n'_{j+1} T'_{j+1})
                  - 3/2 ((n' D_eps T')_{j+1} - (n' D_eps T')_j)/dx + dH_{j+1/2},
      P_j = -(Gamma_{j+1/2} E_{j+1/2} + Gamma_{j-1/2} E_{j-1/2}) / 2;
 4. T' clamped to the table's range.
g, h, dnu are optional closure corrections per cell (flux per electron,
energy flux per electron, ionization frequency).  The two flux corrections
enter implicitly, as first-order upwind advection by the face velocities
gf = (g_j + g_{j+1}) / 2 and wf = (w_j + w_{j+1}) / 2, w = h / T (T of the
step's start): dG_{j+1/2} = max(gf, 0) n'_j + min(gf, 0) n'_{j+1} is part of
the continuity matrix (and of Gamma in step 2), dH_{j+1/2} =
max(wf, 0) n'_j T'_j + min(wf, 0) n'_{j+1} T'_{j+1} part of the energy matrix.
Backward-Euler upwind advection keeps the continuity matrix an M-matrix: n'
stays positive at any time step, where central differences of a cell-to-cell
varying g do not.
With pair losses (col["pair"] true) nu_w = sum(n (nu_i + dnu)) / sum(n) at the
step's start: the continuum form of the particle model's pair losses.
Table lookup: x = (T - T0)/dT clamped to [0, nT - 1], i = min(floor x, nT - 2),
q = q_i + (x - i)(q_{i+1} - q_i), L' = (L_{i+1} - L_i)/dT.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spl

TD = 1e-21
QE = 1.602176634e-19
NAMES = ("muN", "DN", "mueN", "DeN", "nu_izN", "lossN")


def make_table(records, nT: int) -> dict:
    """Resample transport records (dicts with mean_eps_eV and the per-N
    quantities, Te = 2/3 mean energy increasing) onto a uniform Te grid."""
    Te = np.array([2.0 / 3.0 * r["mean_eps_eV"] for r in records])
    if np.any(np.diff(Te) <= 0):
        raise ValueError("Te must increase along the records")
    grid = np.linspace(Te[0], Te[-1], nT)
    tab = {k: np.interp(grid, Te, np.array([r[k] for r in records])) for k in NAMES}
    tab["T0"], tab["dT"], tab["nT"] = grid[0], grid[1] - grid[0], nT
    return tab


def lookup(tab, T):
    nT = tab["nT"]
    x = np.clip((T - tab["T0"]) / tab["dT"], 0.0, nT - 1.0)
    i = np.minimum(np.floor(x).astype(int), nT - 2)
    f = x - i
    out = {k: tab[k][i] + f * (tab[k][i + 1] - tab[k][i]) for k in NAMES}
    out["dlossN"] = (tab["lossN"][i + 1] - tab["lossN"][i]) / tab["dT"]
    return out


def cyclic_solve(lo, dg, up, rhs):
    """Row j: lo_j x_{j-1} + dg_j x_j + up_j x_{j+1} = rhs_j, indices mod N."""
    N = len(dg)
    j = np.arange(N)
    A = sp.coo_matrix((np.concatenate([lo, dg, up]),
                       (np.concatenate([j, j, j]), np.concatenate([(j - 1) % N, j, (j + 1) % N]))),
                      shape=(N, N)).tocsc()
    return spl.spsolve(A, rhs)


def coefficients(col, tab, T):
    Ng = col["N_gas"]
    q = lookup(tab, T)
    mu_i = col["mu_iN"] / Ng
    c = dict(mu_e=q["muN"] / Ng, D_e=q["DN"] / Ng, mu_eps=q["mueN"] / Ng, D_eps=q["DeN"] / Ng,
             nu_i=q["nu_izN"] * Ng, L=q["lossN"] * Ng, dL=q["dlossN"] * Ng, mu_i=mu_i)
    c["a"] = mu_i / (c["mu_e"] + mu_i)
    c["b"] = c["mu_e"] / (c["mu_e"] + mu_i)
    return c


def face(v):
    """(v_j + v_{j+1}) / 2 at face j+1/2."""
    return 0.5 * (v + np.roll(v, -1))


def flux_and_field(col, c, n):
    """Gamma and E at faces j+1/2 for density n (eqs. 11 and 10 + 12)."""
    dx = col["L_m"] / len(n)
    GT = col["Gamma_T"]
    nD = n * c["D_e"]
    Gam = -face(c["a"]) * (np.roll(nD, -1) - nD) / dx - face(c["b"]) * GT
    nf = face(n)
    E = -(np.roll(nD, -1) - nD) / (dx * nf * face(c["mu_e"])) + GT / (nf * face(c["mu_e"] + c["mu_i"]))
    return Gam, E


def step(col, tab, n, T, dt, corr=None):
    """One step of the scheme; returns (n', T')."""
    N = len(n)
    dx = col["L_m"] / N
    GT, nu_w = col["Gamma_T"], col["nu_w"]
    c = coefficients(col, tab, T)
    g = w = None
    nu_i = c["nu_i"]
    if corr is not None:
        g = corr[0]                # flux per electron: a velocity
        w = corr[1] / T            # energy flux per electron over T: a velocity
        nu_i = nu_i + corr[2]
    if col.get("pair"):      # as many electrons leave as are created, uniformly per electron
        nu_w = np.sum(n * nu_i) / np.sum(n)
    # 1. continuity
    r = dt / dx ** 2
    af = face(c["a"])            # a_{j+1/2}
    am = np.roll(af, 1)          # a_{j-1/2}
    D = c["D_e"]
    lo = -r * am * np.roll(D, 1)
    dg = 1.0 + r * (af + am) * D + dt * nu_w
    up = -r * af * np.roll(D, -1)
    bf = face(c["b"])
    rhs = n + dt / dx * (bf - np.roll(bf, 1)) * GT + dt * n * nu_i
    if g is not None:             # + dt/dx (dG_{j+1/2} - dG_{j-1/2}) on the left, upwind
        gp, gm = np.maximum(face(g), 0.0), np.minimum(face(g), 0.0)     # at faces j+1/2
        lo = lo - dt / dx * np.roll(gp, 1)
        dg = dg + dt / dx * (gp - np.roll(gm, 1))
        up = up + dt / dx * gm
    n1 = cyclic_solve(lo, dg, up, rhs)
    # 2. flux and field from n'
    Gam, E = flux_and_field(col, c, n1)
    if g is not None:
        Gam = Gam + gp * n1 + gm * np.roll(n1, -1)
    P = -0.5 * (Gam * E + np.roll(Gam * E, 1))
    # 3. energy
    s = dt / dx
    mef = face(c["mu_eps"])
    Ep, Em = E, np.roll(E, 1)
    mep, mem = mef, np.roll(mef, 1)
    De = c["D_eps"]
    k = 1.5 / dx
    dg = 1.5 * n1 + dt * n1 * c["dL"] + s * (-0.75 * mep * Ep + 0.75 * mem * Em) * n1 + 2.0 * s * k * n1 * De
    up = s * (-0.75 * mep * Ep - k * np.roll(De, -1)) * np.roll(n1, -1)
    lo = s * (0.75 * mem * Em - k * np.roll(De, 1)) * np.roll(n1, 1)
    rhs = 1.5 * n * T + dt * P - dt * n1 * (c["L"] - c["dL"] * T)
    if w is not None:             # + s (dH_{j+1/2} - dH_{j-1/2}) on the left, upwind
        wp, wm = np.maximum(face(w), 0.0), np.minimum(face(w), 0.0)
        lo = lo - s * np.roll(wp * n1, 1)
        dg = dg + s * (wp - np.roll(wm, 1)) * n1
        up = up + s * wm * np.roll(n1, -1)
    T1 = cyclic_solve(lo, dg, up, rhs)
    T1 = np.clip(T1, tab["T0"], tab["T0"] + (tab["nT"] - 1) * tab["dT"])
    return n1, T1


def modes(n, M):
    """c_m = (1/N) sum_j n_j exp(-2 pi i m j / N), m = 1..M."""
    return np.fft.fft(n)[1:M + 1] / len(n)


def features(col, tab, n, T, step=1):
    """Closure-network inputs per cell j (unnormalised): n/<n>, mean energy 3/2 T [eV] and
    E/N [Td] (E at cells the average of its faces) at cells j + d step, d = -2..2."""
    c = coefficients(col, tab, T)
    _, E = flux_and_field(col, c, n)
    Ec = 0.5 * (E + np.roll(E, 1))
    q = (n / n.mean(), 1.5 * T, Ec / (col["N_gas"] * TD))
    return np.stack([np.roll(v, -d * step) for v in q for d in (-2, -1, 0, 1, 2)], 1)
