"""Build liblb3e.so in-tree for sm_103a (nvcc cross-compiles without a GPU).

Usage: python -m paper_2608_05787_b300.build [--force]
"""
from __future__ import annotations

import os
import subprocess
import sys
from pathlib import Path

HERE = Path(__file__).resolve().parent
CSRC = HERE / "csrc"
INCLUDE = HERE.parent / "include"
LIB = HERE / "liblb3e.so"
BUILD = HERE / "_build"

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", str(INCLUDE), "-I", str(CSRC)]
UNITS = {
    # FP64: no contraction into FMA, so the arithmetic rounds like plain C
    "lb3e_f64.cu": ["--fmad=false"],
    "lb3e_f32.cu": [],
    # the three-dimensional (D3Q15) step, FP64 without contraction and FP32
    "lb3e_3d_f64.cu": ["--fmad=false"],
    "lb3e_3d_f32.cu": [],
    # dual-number (tangent) builds
    "lb3e_tangent.cu": [],
    # fixed-scratch observables for callers that cannot allocate (FP64 like lb3e_f64.cu)
    "lb3e_noalloc.cu": ["--fmad=false"],
    "lb3e_api.cpp": [],
}


def _nvcc() -> str:
    cand = os.environ.get("NVCC") or "/usr/local/cuda/bin/nvcc"
    return cand if Path(cand).exists() else "nvcc"


def sources():
    return sorted(p for p in CSRC.iterdir() if p.suffix in (".cu", ".cuh", ".cpp", ".h")) + \
        [INCLUDE / "lb3e.h"]


def up_to_date() -> bool:
    if not LIB.exists():
        return False
    t = LIB.stat().st_mtime
    return all(s.stat().st_mtime <= t for s in sources())


def build(force: bool = False, verbose: bool = False) -> Path:
    if not force and up_to_date():
        return LIB
    BUILD.mkdir(exist_ok=True)
    nvcc = _nvcc()
    cmds, objs = [], []
    for unit, extra in UNITS.items():
        obj = BUILD / (unit + ".o")
        lang = ["-x", "cu"] if unit.endswith(".cu") else []
        cmds.append([nvcc, *ARCH, *COMMON, *extra, *lang, "-c", str(CSRC / unit), "-o", str(obj)])
        objs.append(str(obj))
    # the translation units are independent: compile them concurrently
    from concurrent.futures import ThreadPoolExecutor

    def run(cmd):
        if verbose:
            print(" ".join(cmd), flush=True)
        subprocess.run(cmd, check=True)

    with ThreadPoolExecutor(max_workers=max(1, min(len(cmds), os.cpu_count() or 1))) as ex:
        for f in [ex.submit(run, c) for c in cmds]:
            f.result()
    tmp = LIB.with_suffix(f".{os.getpid()}.tmp")
    subprocess.run([nvcc, *ARCH, "-shared", "-o", str(tmp), *objs], check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
    print(LIB)
