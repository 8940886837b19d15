"""Builds libpagani_gb300.so for sm_103a from csrc/ (nvcc, one -gencode).

The translation units compile in parallel; the result is written in-tree to
paper_2104_06494_gb300/_build/.  Usage: python -m paper_2104_06494_gb300.build
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libpagani_gb300.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", os.path.join(HERE, "..", "include")]
CU_SOURCES = ["pagani_host.cu", "eval_product_peak.cu", "eval_gaussian.cu", "eval_oscillatory.cu",
              "eval_corner_peak.cu", "eval_c0.cu", "eval_discontinuous.cu", "eval_box_power.cu"]
CPP_SOURCES = ["pagani_rule.cpp"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _sources():
    return [os.path.join(CSRC, s) for s in CU_SOURCES + CPP_SOURCES]


def _units():
    """(source, extra flags, object name): every eval_*.cu is compiled twice,
    the second time with -DPAGANI_GM7 for the degree-7 rule variant."""
    units = []
    for src in _sources():
        base = os.path.basename(src)
        units.append((src, [], base + ".o"))
        if base.startswith("eval_"):
            units.append((src, ["-DPAGANI_GM7"], base[:-3] + "_gm7.cu.o"))
    return units


def _headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    hs.append(os.path.join(HERE, "..", "include", "pagani.h"))
    return hs


def up_to_date() -> bool:
    if not os.path.exists(LIB) or os.environ.get("PAGANI_EXTRA_NVCC_FLAGS"):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(p) <= t for p in _sources() + _headers() + [os.path.abspath(__file__)])


def build(force: bool = False, verbose: bool = False, extra_flags: list[str] | None = None) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(OUT, exist_ok=True)
    nvcc = _nvcc()
    # PAGANI_EXTRA_NVCC_FLAGS: extra nvcc flags for tuning builds (e.g. -DPAGANI_EVAL_MINB=3)
    env_flags = os.environ.get("PAGANI_EXTRA_NVCC_FLAGS", "").split()
    flags = NVCC_FLAGS + env_flags + (extra_flags or [])

    def compile_one(unit) -> str:
        src, defs, name = unit
        obj = os.path.join(OUT, name)
        if src.endswith(".cu"):
            cmd = [nvcc] + flags + defs + ["-c", src, "-o", obj]
        else:
            cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-I", os.path.join(HERE, "..", "include"),
                   "-I", "/usr/local/cuda/include", "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr, file=sys.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, _units()))
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart_static", "-lrt", "-ldl", "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True,
                extra_flags=["-Xptxas", "-v"] if "--ptxas-v" in sys.argv else None))
