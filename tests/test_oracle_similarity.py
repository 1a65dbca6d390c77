"""Similarity pin of the particle oracle (Sec. II: without stepwise ionization and Coulomb
collisions the usual discharge scaling laws hold, and results depend on E0/p, nu/p, Rp, lambda p
and gamma/p).

The kinetic problem is invariant under p -> a p, x -> x/a, t -> t/a, E -> a E, n -> a^2 n, with
velocities and energies unchanged: collision frequencies grow as n_g, so nu dt is unchanged;
Gauss's law dE/dx = e (n_i - n_e)/eps0 holds with both sides scaled by a^2; the kick q E dt/m and
the drift v dt/dx in cell units are unchanged.  With a = 2 every rescaled input differs by an
exact power of two, so a correct implementation follows the same trajectory in cell units bit for
bit: the same cells, offsets, velocities, ids and collision counts, node charges equal and fields
exactly doubled.  A quantity with a wrong dimension (a macro-weight with the wrong power of the
length, a dt missing from a probability, dx in place of L) breaks this."""
import numpy as np
import pytest

import oracle
from paper_2202_03215_gb300 import workloads as w


def scaled(p: w.Params, a: float) -> w.Params:
    """The similar column: pressure x a, lengths / a, time step / a, density x a^2, applied
    field x a (a fixed voltage over the shorter column gives it), wall-loss frequency x a."""
    return p.with_(pressure_torr=p.pressure_torr * a, L_m=p.L_m / a, R_m=p.R_m / a, dt_s=p.dt_s / a,
                   n0_m3=p.n0_m3 * a * a, E0_Vpm=p.E0_Vpm * a, nu_w=p.nu_w * a)


SAME = ("cell_e", "off_e", "vx_e", "vy_e", "vz_e", "id_e", "cell_i", "off_i", "vx_i", "vy_i", "vz_i", "id_i",
        "Q_e", "Q_i")


def assert_similar(s1: dict, s2: dict, a: float, what: str) -> None:
    assert s1["n_e"] == s2["n_e"] and s1["n_i"] == s2["n_i"], what
    for k in SAME:
        assert np.array_equal(s1[k], s2[k]), f"{what}: {k}"
    assert np.array_equal(s2["E"], a * s1["E"]), f"{what}: E"


CASES = {
    # argon, 20 V over the column, paired losses, FP64 storage
    "argon_pair_fp64": dict(f32=False, p=w.config_argon_small(seed=5, n_e0=3000, n_i0=3000)),
    # the same in the FP32 storage form
    "argon_pair_fp32": dict(f32=True, p=w.config_argon_small(seed=6, n_e0=3000, n_i0=3000, precision=w.MIXED)),
    # neon at an imposed field with radial losses at nu_w (a non-neutral column: background charge)
    "neon_radial": dict(f32=False, p=w.config_neon_column(seed=7, precision=w.FP64, n_per_species=3000,
                                                         n_cells=256, L_m=0.02, E0_Vpm=1500.0,
                                                         loss_mode=w.LOSS_RADIAL, nu_w=2e7, sort_every=0)),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_similar_columns_follow_the_same_trajectory(case):
    c = CASES[case]
    p1 = c["p"]
    p2 = scaled(p1, 2.0)
    o1, o2 = oracle.Oracle(p1, f32=c["f32"]), oracle.Oracle(p2, f32=c["f32"])
    d1, d2 = o1.derived(), o2.derived()
    assert d2["n_g"] == 2 * d1["n_g"] and d2["dx"] == d1["dx"] / 2 and d2["w"] == 2 * d1["w"]
    assert d2["P_null_e"] == d1["P_null_e"] and d2["P_null_i"] == d1["P_null_i"]
    assert d2["nu_star_e"] == 2 * d1["nu_star_e"]
    assert_similar(o1.get_state(), o2.get_state(), 2.0, "init")
    for n in (1, 9, 50):   # 60 steps in all: six ion pushes, births, losses
        o1.step(n)
        o2.step(n)
        assert_similar(o1.get_state(), o2.get_state(), 2.0, f"{case} step {o1.get_state()['step']}")
    s1, s2 = o1.stats(), o2.stats()
    assert s1["n_coll_e"] == s2["n_coll_e"] and s1["n_coll_i"] == s2["n_coll_i"]
    assert sum(s1["n_coll_e"]) > 0 and sum(s1["n_coll_i"]) > 0


def test_similar_columns_moments_scale():
    """Diagnostic moments of similar columns: densities and fluxes x a^2 (per volume), mean energy
    unchanged, the ionization rate per volume x a^3, the field x a, the potential unchanged."""
    p1 = w.config_argon_small(seed=8, n_e0=3000, n_i0=3000, diag_every=1)
    p2 = scaled(p1, 2.0)
    o1, o2 = oracle.Oracle(p1), oracle.Oracle(p2)
    o1.step(30)
    o2.step(30)
    m1, m2 = o1.moments(), o2.moments()
    assert m1["n_samples"] == m2["n_samples"] > 0
    for k, f in (("n_e", 4.0), ("n_i", 4.0), ("gamma_e", 4.0), ("heat_e", 4.0), ("gamma_i", 4.0),
                 ("mean_eps_e", 1.0), ("iz_rate", 8.0), ("E", 2.0), ("phi", 1.0)):
        assert np.array_equal(m2[k], f * m1[k]), k
    assert m1["iz_rate"].sum() > 0
