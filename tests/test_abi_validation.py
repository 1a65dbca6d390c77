"""Host-side parameter checks of pic_init through the C ABI: every invalid problem statement is
rejected with PIC_EINVAL and a message before any device call, so these run without a GPU."""
import numpy as np
import pytest

import paper_2202_03215_gb300 as pb
from paper_2202_03215_gb300 import build as pbuild
from paper_2202_03215_gb300 import workloads as w


@pytest.fixture(scope="module", autouse=True)
def _built():
    pbuild.build()


def _ok(**kw):
    base = dict(n_e0=1000, n_i0=1000)
    base.update(kw)
    return w.config_argon_small(**base)


def _bad_xsec(kind=w.ELASTIC, energies=(0.0, 10.0), sigmas=(1e-19, 1e-19)):
    return w.XSec(kind, np.array(energies, float), np.array(sigmas, float))


CASES = {
    "two cells": (_ok(n_cells=2), "n_cells"),
    "too many cells": (_ok(n_cells=70000), "n_cells"),
    "zero time step": (_ok(dt_s=0.0), "dt and L"),
    "negative length": (_ok(L_m=-0.05), "dt and L"),
    "negative count": (_ok(n_e0=-1), "negative particle count"),
    "short table": (_ok(n_table=2), "n_table"),
    "storage form": (_ok(precision=7), "precision"),
    "loss mode": (_ok(loss_mode=9), "loss mode"),
    "drive": (_ok(drive=9), "drive"),
    "circuit without field": (_ok(drive=w.DRIVE_CIRCUIT, field_mode=w.FIELD_APPLIED), "circuit"),
    "field mode": (_ok(field_mode=5), "field mode"),
    "ion subcycle": (_ok(ion_subcycle=-1), "ion_subcycle"),
    "bounded with pair losses": (_ok(flags=w.FLAG_BOUNDED, loss_mode=w.LOSS_PAIR), "bounded"),
    "bounded negative emission": (_ok(flags=w.FLAG_BOUNDED, loss_mode=w.LOSS_NONE, J_emit_Am2=-1.0), "emission"),
    "diagnostic period": (_ok(diag_every=7, ion_subcycle=10), "multiple of ion_subcycle"),
    "process kind": (_ok(xsec=[_bad_xsec(kind=9)]), "bad cross section"),
    "descending energies": (_ok(xsec=[_bad_xsec(energies=(10.0, 0.0))]), "not ascending"),
    "seventeen processes": (_ok(xsec=[_bad_xsec()] * 17), "at most 16"),
    "no density": (_ok(n0_m3=0.0), "n0"),
    "energy range": (_ok(eps_max_e_eV=0.0), "eps_max"),
    "column index": (_ok(column=5000), "column"),
    "capacity below the count": (_ok(capacity=10), "capacity"),
    "infinite field": (_ok(drive=w.DRIVE_E0, E0_Vpm=float("inf")), "E0_Vpm is not finite"),
    "NaN pressure": (_ok(pressure_torr=float("nan")), "pressure_torr is not finite"),
    "NaN radius, (R, I) drive": (_ok(drive=w.DRIVE_RI, I_A=1e-3, R_m=float("nan")), "R_m is not finite"),
    "gas temperature": (_ok(T_gas_K=0.0), "gas mass and temperature"),
    "gas mass": (_ok(gas_mass_amu=-4.0), "gas mass and temperature"),
    "negative pressure": (_ok(pressure_torr=-1.0), "pressure"),
    "negative initial temperature": (_ok(Te0_eV=-1.0), "initial temperatures"),
    "negative loss frequency": (_ok(loss_mode=w.LOSS_RADIAL, nu_w=-1.0), "nu_w"),
    "NaN cross section": (_ok(xsec=[_bad_xsec(sigmas=(1e-19, float("nan")))]), "non-finite value"),
    "negative cross section": (_ok(xsec=[_bad_xsec(sigmas=(1e-19, -1e-20))]), "negative"),
    "negative threshold": (_ok(xsec=[w.XSec(w.EXCITATION, np.array([0.0, 20.0]), np.array([0.0, 1e-20]), -5.0)]),
                           "threshold"),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_invalid_problem_is_rejected_before_the_device(case):
    p, msg = CASES[case]
    with pytest.raises(pb.PicError) as ei:
        pb.Column(p)
    assert ei.value.code == -1, str(ei.value)
    assert msg in str(ei.value)


def test_sixteen_processes_pass_the_checks():
    """The limit itself is accepted by the checks (what follows needs a device)."""
    p = _ok(xsec=[_bad_xsec()] * 16, n_e0=0, n_i0=0)
    try:
        pb.Column(p).close()
    except pb.PicError as e:
        assert e.code != -1, str(e)   # without a GPU: a CUDA error, not a parameter error
