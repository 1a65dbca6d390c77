"""Parity of the CUDA path with the CPU oracle, through the C ABI.

From an identical state, everything a step decides is bit-exact: cells,
offsets, velocities, ids, per-particle process codes, fixed-point node
charges, births, removals, victim slots, particle counts.  The field is
bit-exact too (exact integer Gauss-law numerator, one correctly rounded
conversion on both sides); the moments, which the GPU accumulates with
floating-point atomics in arbitrary order, agree to 1e-9 relative.
"""
import numpy as np
import pytest

import oracle
import paper_2202_03215_gb300 as pb
from paper_2202_03215_gb300 import build as pbuild
from paper_2202_03215_gb300 import workloads as w
from tests.helpers import QE, ME, beam_state

pytestmark = pytest.mark.gpu

STATE_KEYS = ("cell_e", "off_e", "vx_e", "vy_e", "vz_e", "id_e",
              "cell_i", "off_i", "vx_i", "vy_i", "vz_i", "id_i", "Q_e", "Q_i", "E")


@pytest.fixture(scope="module", autouse=True)
def _built():
    pbuild.build()


def assert_same(g, o, where=""):
    for k in ("n_e", "n_i", "step", "next_id"):
        assert g[k] == o[k], (where, k, g[k], o[k])
    for k in STATE_KEYS:
        a, b = g[k], o[k]
        if not np.array_equal(a, b):
            bad = np.nonzero(a != b)[0]
            raise AssertionError(f"{where} {k}: {len(bad)} differ, first {bad[:5]} gpu {a[bad[:3]]} oracle {b[bad[:3]]}")


def small(precision=w.FP64, **kw):
    base = dict(n_e0=20000, n_i0=20000, precision=precision, seed=7)
    base.update(kw)
    return w.config_argon_small(**base)


@pytest.mark.parametrize("precision", [w.FP64, w.MIXED])
def test_initial_state_matches(precision):
    p = small(precision)
    g, o = pb.Column(p), oracle.Oracle(p)
    assert_same(g.get_state(), o.get_state(), "init")
    gd, od = g.derived(), o.derived()
    for k in gd:
        assert gd[k] == od[k], k


@pytest.mark.parametrize("sort_every", [0, 5])
@pytest.mark.parametrize("precision", [w.FP64, w.MIXED])
@pytest.mark.parametrize("loss", [w.LOSS_PAIR, w.LOSS_RADIAL, w.LOSS_NONE])
def test_steps_match_bit_exact(precision, loss, sort_every):
    p = small(precision, loss_mode=loss, nu_w=2e8 if loss == w.LOSS_RADIAL else 0.0,
              capacity=40000, sort_every=sort_every)
    g = pb.Column(p, flags=pb.FLAG_RECORD_CODES)
    o = oracle.Oracle(p)
    for n in (1, 9, 1, 10, 4):
        g.step(n)
        o.step(n)
        sg, so = g.get_state(), o.get_state()
        assert_same(sg, so, f"step {so['step']}")
    ng = sg["n_e"]
    assert np.array_equal(g.codes(0, ng), o.codes(0, ng))
    stg, sto = g.stats(), o.stats()
    for k in ("births", "losses_e", "losses_i", "n_coll_e", "n_coll_i", "overflow_e"):
        assert stg[k] == sto[k], k
    assert stg["births"] > 0
    if loss == w.LOSS_RADIAL:
        assert stg["losses_e"] > 0 and stg["losses_i"] > 0


@pytest.mark.parametrize("precision", [w.FP64, w.MIXED])
def test_single_step_from_set_state_with_codes(precision):
    n = 50_000
    p = w.Params(L_m=0.05, n_cells=97, dt_s=2e-11, drive=w.DRIVE_E0, E0_Vpm=3000.0, n_e0=n, n_i0=n,
                 ion_subcycle=1, loss_mode=w.LOSS_PAIR, precision=precision, seed=11,
                 xsec=w.argon_xsecs(sigma_iso=2e-19))
    g = pb.Column(p, flags=pb.FLAG_RECORD_CODES)
    o = oracle.Oracle(p)
    rng = np.random.default_rng(5)
    st = beam_state(n, p.n_cells, np.sqrt(2 * QE * 40.0 / ME), rng, direction=(1, 2, 3), n_i=n,
                    ion_speed=2000.0, step=123456, float32=precision == w.MIXED)
    st["E0"] = 3000.0
    st["E"] = rng.standard_normal(p.n_cells) * 1e3
    if precision == w.MIXED:
        st["E"] = st["E"].astype(np.float32).astype(np.float64)
    g.set_state(st)
    o.set_state(st)
    assert_same(g.get_state(), o.get_state(), "set")
    g.step(1)
    o.step(1)
    assert_same(g.get_state(), o.get_state(), "step")
    for sp in (0, 1):
        cg, co = g.codes(sp, n), o.codes(sp, n)
        assert np.array_equal(cg, co)
        assert len(np.unique(co)) >= 3


@pytest.mark.parametrize("n_cells", [97, 30000])
def test_ragged_sizes_and_frozen_ions(n_cells):
    # 97 cells: one radix pass (odd, copied back); 30000 cells: three passes, field scratch in global memory
    p = small(n_e0=12345, n_i0=12345, n_cells=n_cells, ion_subcycle=0, capacity=20000, sort_every=3)
    g, o = pb.Column(p), oracle.Oracle(p)
    g.step(7)
    o.step(7)
    assert_same(g.get_state(), o.get_state(), "ragged")


@pytest.mark.parametrize("precision", [w.FP64, w.MIXED])
def test_circuit_drive_matches(precision):
    p = small(precision, drive=w.DRIVE_CIRCUIT, U_src=150.0, R_ext_ohm_m2=2.0, E0_Vpm=1000.0)
    g, o = pb.Column(p), oracle.Oracle(p)
    for n in (1, 10, 12):
        g.step(n)
        o.step(n)
        sg, so = g.get_state(), o.get_state()
        assert sg["E0"] == so["E0"] and sg["E0"] != 1000.0
        assert_same(sg, so, "circuit")


def test_uniform_field_swarm_mode():
    p = small(field_mode=w.FIELD_APPLIED, drive=w.DRIVE_E0, E0_Vpm=5e4, loss_mode=w.LOSS_SWARM,
              n_i0=0, ion_subcycle=0)
    g, o = pb.Column(p), oracle.Oracle(p)
    g.step(30)
    o.step(30)
    assert_same(g.get_state(), o.get_state(), "swarm")
    assert g.stats()["births"] == o.stats()["births"] > 0


@pytest.mark.parametrize("precision", [w.FP64, w.MIXED])
def test_moments_match(precision):
    p = small(precision, diag_every=10)
    g, o = pb.Column(p), oracle.Oracle(p)
    g.step(35)
    o.step(35)
    mg, mo = g.moments(), o.moments()
    assert mg["n_samples"] == mo["n_samples"] == 4
    assert mg["n_steps"] == mo["n_steps"] == 35
    # flux, energy and energy flux are summed per CTA in FP32 shared-memory bins before the FP64
    # node sums: within 1e-5 of each array's largest value (the single-step bound for moments);
    # densities and ionization counts are exact
    for k in pb.MOMENT_NAMES:
        a, b = mg[k], mo[k]
        scale = np.abs(b).max() + 1e-300
        assert np.abs(a - b).max() <= 1e-5 * scale, k
    for k in ("n_e", "n_i", "iz_rate", "E"):
        assert np.array_equal(mg[k], mo[k]) or k == "E", k


def test_int128_conversion_on_device():
    rng = np.random.default_rng(1)
    cases = [0, 1, -1, 2**53 + 1, 2**53 + 3, -(2**53 + 1), 2**64 + 2**11, 2**64 + 2**11 + 1,
             (2**63) * 3 + 1, -(2**100) - 1, 2**120 + 2**67, 2**120 + 2**67 + 2**66, -(2**126) + 12345,
             2**64 - 1, -(2**64), 2**65 + 2**12 + 1]
    cases += [int(x) * int(y) for x, y in rng.integers(-2**62, 2**62, (500, 2))]
    cases += [int(x) << int(s) for x, s in zip(rng.integers(-2**62, 2**62, 300), rng.integers(0, 64, 300))]
    got = pb.i128_to_double(cases)
    want = np.array([float(v) for v in cases])
    assert np.array_equal(got, want)


def test_set_state_rejects_particles_outside_the_grid():
    p = w.config_argon_small(n_e0=5000, n_i0=5000, precision=w.MIXED)
    g = pb.Column(p)
    good = g.get_state()
    for key, k, val in (("off_e", 123, 1.0), ("off_i", 7, -1e-300), ("cell_e", 4000, p.n_cells),
                        ("off_e", 9, np.nextafter(1.0, 0.0))):   # the last one rounds to 1 in FP32
        bad = {kk: (v.copy() if isinstance(v, np.ndarray) else v) for kk, v in good.items()}
        bad[key][k] = val
        with pytest.raises(pb.PicError, match=f"particle {k} of species {0 if key.endswith('_e') else 1}"):
            g.set_state(bad)
    g.set_state(good)
    o = oracle.Oracle(p)
    o.set_state(good)
    g.step(2)
    o.step(2)
    assert_same(g.get_state(), o.get_state(), "after a rejected state")
    g.close()


def test_full_size_neon_column_first_step():
    """The benchmark's neon column (2e7 per species, R = 1 cm carrying I = 1 mA) in its
    launch configuration: the field and density of eq. 2 come from the oracle's own
    two-term solve and are given to both sides; initial state and first step (an ion
    step) bit-exact against the oracle."""
    from oracle import two_term as tt
    p = w.config_neon_column(drive=w.DRIVE_RI, I_A=1e-3)
    xs = [(x.kind, x.threshold_eV, x.energy_eV, x.sigma_m2) for x in p.xsec]
    E0, n0, _ = tt.ri_drive(xs, p.gas_mass_amu, p.pressure_torr, p.T_gas_K, p.R_m, p.I_A, p.eps_max_e_eV)
    p = p.with_(drive=w.DRIVE_E0, E0_Vpm=float(E0), n0_m3=float(n0))
    g = pb.Column(p)
    o = oracle.Oracle(p)
    assert_same(g.get_state(), o.get_state(), "init")
    g.step(1)
    o.step(1)
    assert_same(g.get_state(), o.get_state(), "step 1")
    assert g.stats()["n_coll_e"] == o.stats()["n_coll_e"]


def test_full_size_neon_column_moments():
    """Diagnostic moments of one step (an ion step) of the benchmark's neon column, 2e7 per
    species in 16384 cells: the GPU step sums flux, energy and energy flux per CTA cell window in
    FP32 shared-memory bins (in the field's place, the field then gathered from global memory)
    and the oracle sums every particle in FP64.  Within 1e-5 of each array's largest value;
    densities and ionization counts exact."""
    from oracle import two_term as tt
    p = w.config_neon_column(drive=w.DRIVE_RI, I_A=1e-3)
    xs = [(x.kind, x.threshold_eV, x.energy_eV, x.sigma_m2) for x in p.xsec]
    E0, n0, _ = tt.ri_drive(xs, p.gas_mass_amu, p.pressure_torr, p.T_gas_K, p.R_m, p.I_A, p.eps_max_e_eV)
    p = p.with_(drive=w.DRIVE_E0, E0_Vpm=float(E0), n0_m3=float(n0), diag_every=10)   # step 0 is sampled
    g = pb.Column(p)
    o = oracle.Oracle(p)
    g.step(1)
    o.step(1)
    mg, mo = g.moments(), o.moments()
    g.close()
    rel = {}
    for k in pb.MOMENT_NAMES:
        a, b = mg[k], mo[k]
        rel[k] = float(np.abs(a - b).max() / (np.abs(b).max() + 1e-300))
    print("largest difference / largest value:", rel)
    assert all(v <= 1e-5 for v in rel.values()), rel
    for k in ("n_e", "n_i", "iz_rate"):
        assert np.array_equal(mg[k], mo[k]), k


@pytest.mark.parametrize("precision", [w.FP64, w.MIXED])
def test_set_state_f32_equals_set_state(precision):
    """pic_set_state_f32 (FP32 offsets and velocities, the precision form's storage) installs
    the state pic_set_state installs from the same values in FP64: particles, charges and field
    bit for bit, and the same trajectory after it; an offset of 1 in FP32 is refused alike."""
    p = small(precision)
    g = pb.Column(p)
    g.step(7)
    st = g.get_state()
    st32, st64 = dict(st), dict(st)
    for k in ("off", "vx", "vy", "vz"):
        for sp in ("e", "i"):
            st32[f"{k}_{sp}"] = st[f"{k}_{sp}"].astype(np.float32)
            st64[f"{k}_{sp}"] = st32[f"{k}_{sp}"].astype(np.float64)
    a, b = pb.Column(p), pb.Column(p)
    a.set_state(st64)
    b.set_state(st32)
    assert_same(a.get_state(), b.get_state(), "set")
    a.step(12)
    b.step(12)
    assert_same(a.get_state(), b.get_state(), "12 steps after")
    bad = dict(st32)
    bad["off_e"] = st32["off_e"].copy()
    bad["off_e"][5] = np.float32(1.0)
    with pytest.raises(pb.PicError, match="particle 5 of species 0"):
        b.set_state(bad)
    for c in (g, a, b):
        c.close()
