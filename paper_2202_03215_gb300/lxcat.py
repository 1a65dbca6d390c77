"""Cross-section sets in the LXCat text format, read into the process lists a column takes.

The paper draws its electron-neutral cross sections from LXCat databases (Sec. II); none ship
with this package, so the workloads use synthetic shapes (`workloads.py`).  This module lets a
user bring a set downloaded from LXCat.

The format, as LXCat writes it: free text, then one block per process.  A block opens with a
line holding only the process keyword (ELASTIC, EFFECTIVE, MOMENTUM, EXCITATION, IONIZATION or
ATTACHMENT), followed by a line naming the target (or the reaction) and, except for ATTACHMENT,
a line whose first number is the electron-to-target mass ratio (ELASTIC, EFFECTIVE, MOMENTUM) or
the threshold in eV (EXCITATION, IONIZATION).  Lines of the form "KEY: value" follow (SPECIES,
PROCESS, PARAM., COMMENT, UPDATED, COLUMNS), then the table between two lines of dashes: energy in
eV and cross section in m^2, one pair per line.

Mapping onto the model (Sec. II; all electron scattering isotropic):
  ELASTIC                 -> ELASTIC
  EFFECTIVE / MOMENTUM    -> ELASTIC with the inelastic cross sections taken out: with isotropic
                             scattering an inelastic event transfers, on average, all of the
                             electron's momentum, so sigma_el = sigma_m - sum of the inelastic
                             sigmas (clipped at zero), on the union of the energy grids
  EXCITATION              -> EXCITATION (threshold from the block; a second number, the ratio of
                             statistical weights, is ignored: no superelastic collisions)
  IONIZATION              -> IONIZATION
  ATTACHMENT              -> not in the model (rare gases); an error unless dropped
Interpolation follows the library's rule: linear between points, the end values held outside,
excitation and ionization zero below threshold.
"""
from __future__ import annotations

import re
from dataclasses import dataclass, field
from typing import Dict, Iterable, List, Optional

import numpy as np

from . import workloads as w

KEYWORDS = ("ELASTIC", "EFFECTIVE", "MOMENTUM", "EXCITATION", "IONIZATION", "ATTACHMENT")
_MASS_RATIO = ("ELASTIC", "EFFECTIVE", "MOMENTUM")
_INELASTIC = ("EXCITATION", "IONIZATION")
MAX_PROCESSES = 16   # per species, as the library's tables allow


@dataclass
class Record:
    """One block of an LXCat file."""
    keyword: str
    target: str
    param: Optional[float]            # mass ratio or threshold (eV); None for ATTACHMENT
    energy_eV: np.ndarray
    sigma_m2: np.ndarray
    info: Dict[str, str] = field(default_factory=dict)

    @property
    def species(self) -> str:
        """The target species: from "SPECIES: e / Ar" if given, else the first word of the target
        line ("Ar", or "Ar" from "Ar -> Ar*")."""
        sp = self.info.get("SPECIES", "")
        if "/" in sp:
            return sp.split("/", 1)[1].strip()
        return self.target.split()[0] if self.target.split() else ""


def _is_dashes(line: str) -> bool:
    s = line.strip()
    return len(s) >= 5 and set(s) == {"-"}


def parse(text: str) -> List[Record]:
    """All process blocks of an LXCat text, in file order.  Raises ValueError (with the line
    number) on a block without its number line, an unterminated table, a row that is not two
    numbers, descending energies or a negative cross section."""
    lines = text.splitlines()
    out: List[Record] = []
    i, n = 0, len(lines)
    while i < n:
        key = lines[i].strip()
        if key not in KEYWORDS:
            i += 1
            continue
        if i + 1 >= n:
            raise ValueError(f"line {i + 1}: {key} block ends after its keyword")
        target = lines[i + 1].strip()
        j = i + 2
        param = None
        if key != "ATTACHMENT":
            tok = lines[j].split() if j < n else []
            try:
                param = float(tok[0])
            except (IndexError, ValueError):
                raise ValueError(f"line {j + 1}: {key} block '{target}' needs its "
                                 f"{'mass ratio' if key in _MASS_RATIO else 'threshold'}") from None
            j += 1
        info: Dict[str, str] = {}
        while j < n and not _is_dashes(lines[j]):
            m = re.match(r"\s*([A-Z][A-Z0-9 .]*?)\s*:\s?(.*)$", lines[j])
            if m and m.group(1) not in info:
                info[m.group(1)] = m.group(2).strip()
            j += 1
        if j >= n:
            raise ValueError(f"{key} block '{target}' (line {i + 1}): no table")
        start = j + 1
        j = start
        rows = []
        while j < n and not _is_dashes(lines[j]):
            s = lines[j].split()
            if s:
                try:
                    if len(s) < 2:
                        raise ValueError
                    rows.append((float(s[0]), float(s[1])))
                except ValueError:
                    raise ValueError(f"line {j + 1}: not an energy and a cross section: {lines[j]!r}") from None
            j += 1
        if j >= n:
            raise ValueError(f"{key} block '{target}' (line {i + 1}): table not closed by dashes")
        if not rows:
            raise ValueError(f"{key} block '{target}' (line {i + 1}): empty table")
        e = np.array([r[0] for r in rows], dtype=np.float64)
        sg = np.array([r[1] for r in rows], dtype=np.float64)
        if np.any(np.diff(e) < 0):
            raise ValueError(f"{key} block '{target}' (line {i + 1}): energies not ascending")
        if np.any(sg < 0) or not np.all(np.isfinite(sg)) or not np.all(np.isfinite(e)):
            raise ValueError(f"{key} block '{target}' (line {i + 1}): negative or non-finite values")
        cols = info.get("COLUMNS", "").lower().replace(" ", "")
        if "cm2" in cols or "cm^2" in cols:
            sg = sg * 1e-4
        out.append(Record(key, target, param, e, sg, info))
        i = j + 1
    return out


def sigma_at(x: w.XSec, eps: np.ndarray) -> np.ndarray:
    """sigma of a process at energies eps by the library's rule: linear between points, the end
    values held outside, zero below threshold for excitation and ionization."""
    s = np.interp(eps, x.energy_eV, x.sigma_m2)
    if x.kind in (w.EXCITATION, w.IONIZATION):
        s = np.where(eps < x.threshold_eV, 0.0, s)
    return s


def electron_xsecs(records: Iterable[Record], species: Optional[str] = None,
                   drop_attachment: bool = False) -> List[w.XSec]:
    """The electron-neutral process list of one target, in the order the model uses: elastic,
    excitation levels by ascending threshold, ionization."""
    recs = [r for r in records if species is None or r.species == species]
    if species is None and len({r.species for r in recs}) > 1:
        raise ValueError(f"several targets {sorted({r.species for r in recs})}: name one")
    el = [r for r in recs if r.keyword in _MASS_RATIO]
    if len(el) != 1:
        raise ValueError(f"need exactly one ELASTIC, EFFECTIVE or MOMENTUM block, found {len(el)}")
    att = [r for r in recs if r.keyword == "ATTACHMENT"]
    if att and not drop_attachment:
        raise ValueError("ATTACHMENT is not part of the model; pass drop_attachment=True to leave it out")
    inel = [w.XSec(w.EXCITATION if r.keyword == "EXCITATION" else w.IONIZATION, r.energy_eV.copy(),
                   r.sigma_m2.copy(), float(r.param))
            for r in recs if r.keyword in _INELASTIC]
    exc = sorted((x for x in inel if x.kind == w.EXCITATION), key=lambda x: x.threshold_eV)
    ion = [x for x in inel if x.kind == w.IONIZATION]
    if len(ion) > 1:
        raise ValueError(f"{len(ion)} IONIZATION blocks: the model takes one")
    r0 = el[0]
    if r0.keyword == "ELASTIC":
        elastic = w.XSec(w.ELASTIC, r0.energy_eV.copy(), r0.sigma_m2.copy())
    else:
        grid = np.unique(np.concatenate([r0.energy_eV] + [x.energy_eV for x in inel]
                                        + [np.array([x.threshold_eV]) for x in inel]))
        sm = np.interp(grid, r0.energy_eV, r0.sigma_m2)
        for x in inel:
            sm = sm - sigma_at(x, grid)
        elastic = w.XSec(w.ELASTIC, grid, np.maximum(sm, 0.0))
    out = [elastic] + exc + ion
    if len(out) > MAX_PROCESSES:
        raise ValueError(f"{len(out)} electron processes; the library takes at most {MAX_PROCESSES} "
                         "(lump excitation levels first)")
    return out


def ion_xsec(record: Record, kind: int, frame: str = "lab", mass_ratio_target_over_ion: float = 1.0) -> w.XSec:
    """An ion-neutral process (kind ION_CX or ION_ISO) from a table of cross section against ion
    energy.  The library's ion tables are in the lab-frame energy of an ion hitting a neutral at
    rest, 0.5 M g^2 / e; a table in centre-of-mass energy is converted by
    eps_lab = eps_cm (M_ion + M_target) / M_target."""
    if kind not in (w.ION_CX, w.ION_ISO):
        raise ValueError("kind must be ION_CX or ION_ISO")
    e = record.energy_eV.copy()
    if frame == "cm":
        e = e * (1.0 + 1.0 / mass_ratio_target_over_ion)
    elif frame != "lab":
        raise ValueError("frame must be 'lab' or 'cm'")
    return w.XSec(kind, e, record.sigma_m2.copy())


def format_records(xsecs: Iterable[w.XSec], target: str, mass_ratio: float) -> str:
    """An electron process list written as LXCat text (ELASTIC, EXCITATION, IONIZATION blocks, full
    precision), e.g. to hand a synthetic set to another code; `parse` reads it back exactly."""
    names = {w.ELASTIC: "ELASTIC", w.EXCITATION: "EXCITATION", w.IONIZATION: "IONIZATION"}
    parts = [f"Process list of {target} written by paper_2202_03215_gb300.lxcat", ""]
    for x in xsecs:
        if x.kind not in names:
            raise ValueError("only electron processes are written")
        key = names[x.kind]
        if x.kind == w.ELASTIC:
            head = [key, target, f" {mass_ratio!r}"]
        else:
            head = [key, f"{target} -> {target}*" if x.kind == w.EXCITATION else f"{target} -> {target}^+",
                    f" {float(x.threshold_eV)!r}"]
        parts += head + [f"SPECIES: e / {target}", "COLUMNS: Energy (eV) | Cross section (m2)", "-----------------------------"]
        parts += [f" {float(a)!r}\t{float(b)!r}" for a, b in zip(x.energy_eV, x.sigma_m2)]
        parts += ["-----------------------------", ""]
    return "\n".join(parts) + "\n"
