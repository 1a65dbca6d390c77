"""T2/T3 pins of the oracle's push, deposit and field: exact leapfrog motion
in a constant field, and the cold-plasma oscillation frequency of the
leapfrog scheme, sin(w dt/2) = w_pe dt/2."""
import numpy as np

import oracle
from paper_2202_03215_gb300 import workloads as w
from tests.helpers import AMU, QE, ME, EPS0


def test_constant_field_positions_are_exact_quadratics():
    N, L, dt, E0 = 100, 0.01, 2e-11, 1000.0
    p = w.Params(L_m=L, n_cells=N, dt_s=dt, xsec=[], field_mode=w.FIELD_APPLIED, drive=w.DRIVE_E0,
                 E0_Vpm=E0, n_e0=2000, n_i0=0, ion_subcycle=0, loss_mode=w.LOSS_NONE, Te0_eV=1.0)
    o = oracle.Oracle(p)
    s0 = o.get_state()
    dx = L / N
    x0 = s0["cell_e"] + s0["off_e"]
    v_half = s0["vx_e"]
    a = QE * E0 / ME  # E = -E0, electron charge -e
    for n in (1, 5, 40):
        o.step(n - o.stats()["step"])
        s = o.get_state()
        disp = (n * dt * v_half + a * dt * dt * n * (n + 1) / 2) / dx
        d = (s["cell_e"] + s["off_e"]) - (x0 + disp)
        d = (d + N / 2) % N - N / 2
        assert np.abs(d).max() < 1e-7
        # transverse velocities never change without collisions
        assert np.array_equal(s["vy_e"], s0["vy_e"]) and np.array_equal(s["vz_e"], s0["vz_e"])
    # velocity is exact: v^{n-1/2} = v^{-1/2} + n a dt
    assert np.allclose(s["vx_e"], v_half + 40 * a * dt, rtol=1e-12, atol=1e-6)


def test_cold_plasma_oscillation_leapfrog_dispersion():
    N, ppc, dx, dt = 128, 64, 1e-4, 2e-11
    L = N * dx
    wpe_dt = 0.5
    wpe = wpe_dt / dt
    n0 = wpe ** 2 * EPS0 * ME / QE ** 2
    n = N * ppc
    p = w.Params(L_m=L, n_cells=N, dt_s=dt, xsec=[], drive=w.DRIVE_E0, E0_Vpm=0.0, n_e0=n, n_i0=n,
                 n0_m3=n0, ion_subcycle=0, loss_mode=w.LOSS_NONE, Te0_eV=0.0, Ti0_eV=0.0)
    o = oracle.Oracle(p)
    base = (np.arange(n) + 0.5) / ppc                 # quiet start, in cells
    k = 2 * np.pi / N
    xe = base + 1e-2 * np.sin(k * base)
    st = {"cell_e": np.floor(xe).astype(np.int32), "off_e": xe - np.floor(xe),
          "vx_e": np.zeros(n), "vy_e": np.zeros(n), "vz_e": np.zeros(n), "id_e": np.arange(n, dtype=np.uint64),
          "cell_i": np.floor(base).astype(np.int32), "off_i": base - np.floor(base),
          "vx_i": np.zeros(n), "vy_i": np.zeros(n), "vz_i": np.zeros(n),
          "id_i": np.arange(n, 2 * n, dtype=np.uint64), "step": 0, "next_id": 2 * n, "E0": 0.0,
          "E": None, "Q_i": None}
    o.set_state(st)
    j0 = N // 4  # E is proportional to the displacement sin(k x): extreme at L/4
    trace = []
    for _ in range(400):
        o.step(1)
        trace.append(o.get_state()["E"][j0])
    y = np.array(trace)
    s = np.sign(y)
    idx = np.nonzero(s[:-1] * s[1:] < 0)[0]
    t0 = idx + y[idx] / (y[idx] - y[idx + 1])        # linear interpolation of zero crossings
    period = 2 * np.mean(np.diff(t0)) * dt
    w_meas = 2 * np.pi / period
    w_leap = 2 / dt * np.arcsin(wpe_dt / 2)
    assert abs(w_meas / w_leap - 1) < 1.5e-3
    assert abs(w_meas / wpe - 1) > 5e-3   # the leapfrog correction is resolved


def test_subcycled_ions_move_on_their_push_steps_only():
    """Ion subcycling: ions are pushed on steps 0, sub, 2 sub, ... with dt_i = sub dt and stay put
    in between; over m pushes the leapfrog is exact for a constant field (x quadratic in m dt_i)."""
    N, L, dt, E0, sub = 100, 0.01, 2e-11, 5e6, 10
    p = w.Params(L_m=L, n_cells=N, dt_s=dt, xsec=[], field_mode=w.FIELD_APPLIED, drive=w.DRIVE_E0,
                 E0_Vpm=E0, n_e0=0, n_i0=2000, ion_subcycle=sub, loss_mode=w.LOSS_NONE, Ti0_eV=0.5)
    o = oracle.Oracle(p)
    s0 = o.get_state()
    dx, dti = L / N, sub * dt
    x0 = s0["cell_i"] + s0["off_i"]
    v_half = s0["vx_i"]
    a = -QE * E0 / (p.gas_mass_amu * AMU)   # E = -E0, ion charge +e
    prev = None
    for n in (1, 5, 10, 11, 20, 35):
        o.step(n - o.stats()["step"])
        s = o.get_state()
        m = -(-n // sub)   # pushes on steps 0, sub, ... below n
        disp = (m * dti * v_half + a * dti * dti * m * (m + 1) / 2) / dx
        d = (s["cell_i"] + s["off_i"]) - (x0 + disp)
        d = (d + N / 2) % N - N / 2
        assert np.abs(d).max() < 1e-7, n
        assert np.allclose(s["vx_i"], v_half + m * a * dti, rtol=1e-12, atol=1e-9)
        if prev is not None and prev[0] == m:
            assert np.array_equal(s["cell_i"], prev[1]) and np.array_equal(s["off_i"], prev[2])
        prev = (m, s["cell_i"], s["off_i"])
