"""The C-ABI library loads and exports every entry point that include/pic.h
declares, and the Python binding's struct layouts match the C header's
(checked by compiling a layout probe of the header with the host C compiler).
No compute call is made: these tests need no GPU."""
import ctypes as C
import re
import subprocess
from pathlib import Path

import pytest

import paper_2202_03215_gb300 as pb
from paper_2202_03215_gb300 import build as pbuild

ROOT = Path(__file__).resolve().parents[1]
HEADER = ROOT / "include" / "pic.h"


@pytest.fixture(scope="module")
def libpic():
    pbuild.build()
    return pb.lib()


def declared_functions():
    text = re.sub(r"/\*.*?\*/", "", HEADER.read_text(), flags=re.S)
    return sorted(set(re.findall(r"\b(pic_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("pic_init", "pic_step", "pic_moments", "pic_free", "pic_get_state", "pic_set_state",
              "pic_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(libpic):
    missing = [n for n in declared_functions() if not hasattr(libpic, n)]
    assert not missing
    assert libpic.pic_abi_version() == 1


def test_binding_struct_layout_matches_header(tmp_path):
    structs = {"pic_params": pb.Params, "pic_xsec": pb.Xsec, "pic_state": pb.State, "pic_state_f32": pb.StateF32,
               "pic_stats": pb.Stats, "pic_moments_out": pb.MomentsOut, "pic_transport": pb.Transport,
               "pic_fluid_column": pb.FluidColumn}
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"', 'int main(void) {']
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("  return 0; }")
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    for line in filter(None, out):
        cname, field, val = line.split()
        py = structs[cname]
        if field == "size":
            assert C.sizeof(py) == int(val), cname
        else:
            assert getattr(py, field).offset == int(val), (cname, field)


def test_oracle_params_layout_matches_binding():
    import oracle
    for (a, _), (b, _) in zip(oracle.OraParams._fields_, pb.Params._fields_):
        assert a == b
    assert C.sizeof(oracle.OraParams) == C.sizeof(pb.Params)
