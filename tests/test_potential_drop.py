"""Eq. (1): the potential drop over one striation equals E0 lambda, because the space-charge field
averages to zero over a period.  Checked on a synthetic striation field and on the oracle's
self-consistent field (the periodic solve leaves a zero-mean space-charge field, so the drop over
the whole column is E0 L)."""
import numpy as np
import pytest

import oracle
from paper_2202_03215_gb300 import screen
from paper_2202_03215_gb300 import workloads as w


@pytest.mark.parametrize("m", [1, 4, 16])
def test_eq1_on_a_striation_field(m):
    N, L, E0 = 1024, 0.1, 800.0
    dx = L / N
    x = np.arange(N) * dx
    E = -E0 + 3000.0 * np.sin(2 * np.pi * m * x / L + 0.3)     # strong space-charge modulation
    lam_cells = N // m
    for start in (0, 17, lam_cells // 2):
        assert screen.potential_drop(E, dx, lam_cells, start) == pytest.approx(E0 * L / m, rel=1e-9)
    # over half a wavelength the drop depends on the phase: the identity needs a full period
    half = [screen.potential_drop(E, dx, lam_cells // 2, s) for s in (0, lam_cells // 4)]
    assert abs(half[0] - half[1]) > 1e-3 * E0 * L / m


@pytest.mark.parametrize("loss", [w.LOSS_PAIR, w.LOSS_RADIAL])
def test_eq1_over_the_column_on_the_self_consistent_field(loss):
    p = w.config_argon_small(seed=9, n_e0=20000, n_i0=20000, loss_mode=loss,
                             nu_w=5e8 if loss == w.LOSS_RADIAL else 0.0)
    o = oracle.Oracle(p)
    o.step(25)
    s = o.get_state()
    dx = p.L_m / p.n_cells
    E0 = s["E0"]
    assert np.std(s["E"]) > 1e-3 * E0                    # a real space-charge field
    assert screen.potential_drop(s["E"], dx, p.n_cells) == pytest.approx(E0 * p.L_m, rel=1e-10)
