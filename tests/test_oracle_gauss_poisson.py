"""Pins of the Gaussian inverse-CDF table (T9) and the periodic Poisson
solve (T1) of the oracle, against scipy's normal distribution, the
discrete closed form of a sinusoidal charge and the paper's Thomas route."""
import numpy as np
import pytest
from scipy import special, stats

import oracle

EPS0 = 8.8541878128e-12


def test_gauss_table_entries_are_rounded_normal_quantiles():
    T = oracle.gauss_table()
    k = np.arange(1, 4096)
    z = special.ndtri(k / 4096.0)
    # each entry is Phi^-1(k/4096) rounded to FP32: within half an FP32 ulp (+ scipy error)
    ulp = np.spacing(np.abs(z).astype(np.float32)).astype(np.float64)
    assert np.all(np.abs(T[1:4096] - z) <= 0.5 * ulp + 1e-15 * np.abs(z) + 1e-30)
    # end entry: linear piece with the exact conditional mean of the tail
    z1 = special.ndtri(1 / 4096.0)
    m0 = -4096.0 * stats.norm.pdf(z1)
    assert T[0] == np.float32(2 * m0 - z1)
    assert T[4096] == -T[0]
    assert np.all(T[::-1] == -T)


def _sampler_moments(T):
    # exact mean/variance of the piecewise-linear inverse-CDF sampler
    a, b = T[:-1].astype(np.float64), T[1:].astype(np.float64)
    mean = np.mean((a + b) / 2)
    m2 = np.mean((a * a + a * b + b * b) / 3)
    return mean, m2 - mean ** 2


def test_gauss_sampler_moments_and_ks():
    T = oracle.gauss_table()
    mean, var = _sampler_moments(T)
    assert abs(mean) < 1e-12
    assert abs(var - 1.0) < 2e-3  # stated truncation error of the 4096-interval table
    u = (np.arange(200000) + 0.5) / 200000
    g = np.array([oracle.gauss_sample(T, x) for x in u[::7]])
    # stratified uniforms: the sup-distance to Phi is the table's own error (+1/n)
    assert stats.kstest(g, "norm", method="asymp").statistic < 2e-4
    # the sampler is the linear interpolation of the table
    assert oracle.gauss_sample(T, 0.5) == 0.0
    assert oracle.gauss_sample(T, 1.0 / 4096) == pytest.approx(float(T[1]), abs=0)


def test_int128_to_double_rounds_to_nearest_even():
    rng = np.random.default_rng(1)
    cases = [0, 1, -1, 2**53 + 1, 2**53 + 3, -(2**53 + 1), 2**64 + 2**11, 2**64 + 2**11 + 1,
             (2**63) * 3 + 1, -(2**100) - 1, 2**120 + 2**67, 2**120 + 2**67 + 2**66]
    cases += [int(x) * int(y) for x, y in rng.integers(-2**62, 2**62, (200, 2))]
    for v in cases:
        assert oracle.i128_to_double(v) == float(v), v  # Python's int->float is correctly rounded


def _exact_field(D, w=5e8):
    C = 1.602176634e-19 * w / (EPS0 * 2.0**32)
    Qi = np.where(D > 0, D, 0).astype(np.int64)
    Qe = np.where(D < 0, -D, 0).astype(np.int64)
    return oracle.field_exact(Qi, Qe, C), C


@pytest.mark.parametrize("N,m", [(64, 1), (500, 3), (4096, 17)])
def test_poisson_sinusoid_closed_form(N, m):
    dx = 1e-4
    j = np.arange(N)
    A = 2.0**40
    D = np.round(A * np.sin(2 * np.pi * m * j / N)).astype(np.int64)
    Eh, C = _exact_field(D)
    # rho_j = C eps0 D_j / dx; discrete solution phi_j = rho0 dx^2/(eps0 (2-2cos k dx)) sin(k x_j)
    k = 2 * np.pi * m / (N * dx)
    rho = C * EPS0 * D / dx
    rho0 = C * EPS0 * A / dx
    phi = rho0 * dx**2 / (EPS0 * (2 - 2 * np.cos(k * dx))) * np.sin(k * j * dx)
    Eh_cf = -(np.roll(phi, -1) - phi) / dx
    scale = np.abs(Eh_cf).max()
    assert np.abs(Eh - Eh_cf).max() < 1e-9 * scale
    # the paper's route (Thomas on the gauge-pinned tridiagonal system) agrees
    phi_t = oracle.poisson_thomas(rho - rho.mean(), dx)
    Eh_t = -(np.roll(phi_t, -1) - phi_t) / dx
    assert np.abs(Eh - Eh_t).max() < 1e-10 * scale


def test_poisson_random_charge_thomas_and_gauss_law():
    rng = np.random.default_rng(3)
    N, dx = 1000, 1e-4
    Qi = rng.integers(0, 2**44, N)
    Qe = rng.integers(0, 2**44, N)
    C = 1.602176634e-19 * 5e8 / (EPS0 * 2.0**32)
    Eh = oracle.field_exact(Qi, Qe, C)
    D = (Qi - Qe).astype(np.float64)
    rho = C * EPS0 * D / dx
    rho_n = rho - rho.mean()   # uniform neutralising background
    phi_t = oracle.poisson_thomas(rho_n, dx)
    Eh_t = -(np.roll(phi_t, -1) - phi_t) / dx
    scale = np.abs(Eh).max()
    assert np.abs(Eh - Eh_t).max() < 1e-10 * scale
    # Gauss's law with the background, and a zero-mean periodic field
    div = (Eh - np.roll(Eh, 1)) / dx
    assert np.abs(div - rho_n / EPS0).max() < 1e-9 * np.abs(rho_n / EPS0).max()
    assert abs(Eh.mean()) < 1e-12 * scale
