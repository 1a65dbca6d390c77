"""Build the in-tree CUDA library libpic.so for sm_103a with nvcc.

The translation units compile in parallel; the result lands next to this
file.  Kernels are compiled with -fmad=false and host code with
-ffp-contract=off: every floating-point expression of the particle step
rounds as written, which the bit-exact parity with the CPU oracle relies on.
The closure network's sources, checked within BF16 tolerances, may contract.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor
from pathlib import Path

HERE = Path(__file__).resolve().parent
ROOT = HERE.parent
CSRC = HERE / "csrc"
INCLUDE = ROOT / "include"
LIB = HERE / "libpic.so"
BUILD = HERE / "_build"
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-fmad=false", "-prec-div=true", "-prec-sqrt=true",
         "-Xcompiler", "-fPIC,-ffp-contract=off,-fno-fast-math", f"-I{INCLUDE}", f"-I{CSRC}"]
# the closure network's kernels are checked against the oracle within BF16 tolerances, not bit for
# bit, so they may contract multiply-adds; every other source rounds each operation as written
CONTRACT_OK = {"pic_mlp.cu", "pic_mlp_tc.cu", "pic_mlp_train_tc.cu"}
SOURCES = ["pic_kernels.cu", "pic_host.cu", "pic_sort.cu", "pic_mlp.cu", "pic_noalloc.cu", "pic_transport.cu", "pic_fluid.cu",
           "pic_mlp_tc.cu", "pic_mlp_train_tc.cu"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and Path(c).exists():
            return c
    raise RuntimeError("nvcc not found")


def _stale() -> bool:
    if not LIB.exists():
        return True
    t = LIB.stat().st_mtime
    deps = list(CSRC.glob("*")) + [INCLUDE / "pic.h", Path(__file__)]
    return any(d.stat().st_mtime > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None) -> Path:
    if not force and not _stale():
        return LIB
    BUILD.mkdir(exist_ok=True)
    cc = nvcc()
    extra = extra or []

    def compile_one(src: str) -> Path:
        obj = BUILD / (Path(src).stem + ".o")
        flags = FLAGS
        if src in CONTRACT_OK:   # not bit-exact against the oracle: FMA contraction allowed
            flags = [f for f in FLAGS if f != "-fmad=false"] + ["-fmad=true"]
        cmd = [cc, *ARCH, *flags, *extra, "-c", str(CSRC / src), "-o", str(obj)]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    with ThreadPoolExecutor(len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB.with_suffix(".so.tmp")
    cmd = [cc, *ARCH, "-shared", "-o", str(tmp), *map(str, objs)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True,
          extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else None)
    print(LIB)
