"""The LXCat-format reader (host code): block parsing, the effective-to-elastic conversion under
isotropic scattering, error paths, and a round trip of a synthetic set that steps bit for bit like
the set it was written from.  The gas "Zz" and its numbers are made up for these tests."""
import numpy as np
import pytest

import oracle
from paper_2202_03215_gb300 import lxcat
from paper_2202_03215_gb300 import workloads as w

SET = """Synthetic cross sections for the reader's tests (made-up gas Zz, made-up values).
Text before the first block: ignored.

EFFECTIVE
Zz
 2.5e-5
SPECIES: e / Zz
PROCESS: E + Zz -> E + Zz, Effective
PARAM.:  m/M = 0.000025
COMMENT: not a real gas: colons: inside comments.
COLUMNS: Energy (eV) | Cross section (m2)
-----------------------------
 0	1.0e-19
 10	2.0e-19
 20	3.0e-19
 40	3.0e-19
-----------------------------

EXCITATION
Zz -> Zz*(10)
 10  0.5
SPECIES: e / Zz
COLUMNS: Energy (eV) | Cross section (m2)
-----------------------------
 10	0
 20	4.0e-20
 40	2.0e-20
-----------------------------

EXCITATION
Zz -> Zz*(5)
 5
SPECIES: e / Zz
-----------------------------
 5	0
 40	7.0e-20
-----------------------------

IONIZATION
Zz -> Zz^+
 15
SPECIES: e / Zz
-----------------------------
 15	0
 40	1.0e-19
-----------------------------

ATTACHMENT
Zz -> Zz^-
SPECIES: e / Zz
-----------------------------
 0	1e-22
 10	1e-22
-----------------------------
"""


def test_blocks_and_fields():
    recs = lxcat.parse(SET)
    assert [r.keyword for r in recs] == ["EFFECTIVE", "EXCITATION", "EXCITATION", "IONIZATION", "ATTACHMENT"]
    assert [r.param for r in recs] == [2.5e-5, 10.0, 5.0, 15.0, None]
    assert {r.species for r in recs} == {"Zz"}
    assert recs[0].info["PARAM."] == "m/M = 0.000025"
    assert recs[0].info["COMMENT"].startswith("not a real gas: colons")
    assert np.array_equal(recs[1].energy_eV, [10.0, 20.0, 40.0])
    assert np.array_equal(recs[1].sigma_m2, [0.0, 4e-20, 2e-20])


def test_effective_becomes_elastic_without_the_inelastic_part():
    xs = lxcat.electron_xsecs(lxcat.parse(SET), drop_attachment=True)
    assert [x.kind for x in xs] == [w.ELASTIC, w.EXCITATION, w.EXCITATION, w.IONIZATION]
    assert [x.threshold_eV for x in xs[1:]] == [5.0, 10.0, 15.0]   # levels by threshold
    el = xs[0]
    assert np.array_equal(el.energy_eV, [0.0, 5.0, 10.0, 15.0, 20.0, 40.0])
    # worked by hand: at 20 eV, 3e-19 - 4e-20 (level 10) - 3e-20 (level 5: 7e-20 * 15/35)
    # - 2e-20 (ionization: 1e-19 * 5/25); below 5 eV the effective value itself
    expect = {0.0: 1e-19, 5.0: 1.5e-19, 10.0: 2e-19 - 1e-20, 20.0: 3e-19 - 4e-20 - 3e-20 - 2e-20,
              40.0: 3e-19 - 2e-20 - 7e-20 - 1e-19}
    for e, s in expect.items():
        got = el.sigma_m2[list(el.energy_eV).index(e)]
        assert got == pytest.approx(s, rel=1e-12, abs=1e-35), e
    # between grid points the model interpolates the result linearly, as the library does
    assert lxcat.sigma_at(el, np.array([30.0]))[0] == pytest.approx(0.5 * (2.1e-19 + 1.1e-19), rel=1e-12)


def test_elastic_block_is_taken_as_is_and_clipping():
    text = SET.replace("EFFECTIVE\nZz\n", "ELASTIC\nZz\n", 1)
    xs = lxcat.electron_xsecs(lxcat.parse(text), drop_attachment=True)
    assert np.array_equal(xs[0].energy_eV, [0.0, 10.0, 20.0, 40.0])
    assert np.array_equal(xs[0].sigma_m2, [1e-19, 2e-19, 3e-19, 3e-19])
    # an effective cross section smaller than the inelastic sum is clipped at zero
    small = SET.replace(" 40\t3.0e-19\n-----", " 40\t1.0e-19\n-----", 1)
    xs = lxcat.electron_xsecs(lxcat.parse(small), drop_attachment=True)
    assert xs[0].sigma_m2[-1] == 0.0 and np.all(xs[0].sigma_m2 >= 0)


def test_attachment_and_target_choice():
    recs = lxcat.parse(SET)
    with pytest.raises(ValueError, match="ATTACHMENT"):
        lxcat.electron_xsecs(recs)
    other = SET.replace("e / Zz", "e / Yy")
    with pytest.raises(ValueError, match="several targets"):
        lxcat.electron_xsecs(recs + lxcat.parse(other), drop_attachment=True)
    xs = lxcat.electron_xsecs(recs + lxcat.parse(other), species="Yy", drop_attachment=True)
    assert len(xs) == 4


@pytest.mark.parametrize("bad, msg", [
    ("EXCITATION\nZz -> Zz*\nSPECIES: e / Zz\n-----\n 1 2\n-----\n", "threshold"),
    ("ELASTIC\nZz\n 1e-5\n-----\n 0 1e-19\n 10 2e-19\n", "not closed"),
    ("ELASTIC\nZz\n 1e-5\n-----\n 10 1e-19\n 0 2e-19\n-----\n", "ascending"),
    ("ELASTIC\nZz\n 1e-5\n-----\n 0 -1e-19\n-----\n", "negative"),
    ("ELASTIC\nZz\n 1e-5\n-----\n 0 abc\n-----\n", "not an energy"),
    ("ELASTIC\nZz\n 1e-5\n-----\n-----\n", "empty"),
])
def test_malformed_blocks_are_rejected(bad, msg):
    with pytest.raises(ValueError, match=msg):
        lxcat.parse(bad)


def test_square_centimetres_are_converted():
    text = "ELASTIC\nZz\n 1e-5\nCOLUMNS: Energy (eV) | Cross section (cm2)\n-----\n 0 1e-15\n 10 2e-15\n-----\n"
    r = lxcat.parse(text)[0]
    assert np.allclose(r.sigma_m2, [1e-19, 2e-19], rtol=1e-15)


def test_ion_table_in_the_centre_of_mass_frame():
    r = lxcat.parse("ELASTIC\nZz+ / Zz\n 1\n-----\n 0 5e-19\n 2 4e-19\n 10 3e-19\n-----\n")[0]
    x = lxcat.ion_xsec(r, w.ION_CX, frame="cm")
    assert x.kind == w.ION_CX
    assert np.array_equal(x.energy_eV, [0.0, 4.0, 20.0])   # equal masses: eps_lab = 2 eps_cm
    assert np.array_equal(lxcat.ion_xsec(r, w.ION_ISO).energy_eV, r.energy_eV)


def test_round_trip_of_the_neon_set_steps_bit_for_bit():
    ne = w.neon_xsecs()
    elec = [x for x in ne if x.kind in (w.ELASTIC, w.EXCITATION, w.IONIZATION)]
    ions = [x for x in ne if x.kind in (w.ION_CX, w.ION_ISO)]
    text = lxcat.format_records(elec, "Ne", 2.72e-5)
    back = lxcat.electron_xsecs(lxcat.parse(text), species="Ne")
    assert len(back) == len(elec)
    for a, b in zip(elec, back):
        assert a.kind == b.kind and a.threshold_eV == b.threshold_eV
        assert np.array_equal(a.energy_eV, b.energy_eV) and np.array_equal(a.sigma_m2, b.sigma_m2)
    p = w.config_neon_column(precision=w.FP64, n_per_species=4000, n_cells=256, L_m=0.02, E0_Vpm=1500.0,
                             sort_every=0)
    o1, o2 = oracle.Oracle(p), oracle.Oracle(p.with_(xsec=back + ions))
    o1.step(30)
    o2.step(30)
    s1, s2 = o1.get_state(), o2.get_state()
    for k in ("cell_e", "off_e", "vx_e", "id_e", "cell_i", "vx_i", "Q_e", "Q_i", "E"):
        assert np.array_equal(s1[k], s2[k]), k
    assert sum(o1.stats()["n_coll_e"]) > 0
