"""Build liblqcd.so (the C-ABI library) for sm_103a with nvcc.

Each translation unit under csrc/ is compiled in parallel into _build/, then
linked into paper_1701_00426_gb300/liblqcd.so (in tree, git-ignored).
Incremental: a unit is rebuilt when it or any header under csrc/ or include/
is newer than its object.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "liblqcd.so")
# The bounds-checked variant (every neighbour index compared with its extent,
# errors recorded in device words read by lqcd_bounds_errors), for tests.
CHECKED_BUILD = os.path.join(HERE, "_build_checked")
CHECKED_LIB = os.path.join(HERE, "liblqcd_checked.so")
INCLUDE = os.path.join(ROOT, "include")

UNITS = ["api.cu", "deo.cu", "solver.cu", "mrhs.cu", "serve.cu", "noalloc.cu", "rational.cu", "gauge.cu", "shard.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I", INCLUDE, "-I", CSRC]
# Extra preprocessor definitions for tuning builds (e.g. "-DLQCD_TILE_SITES=64").
EXTRA = os.environ.get("LQCD_NVCC_DEFINES", "").split()


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def _headers_mtime() -> float:
    m = 0.0
    for d in (CSRC, INCLUDE):
        for f in os.listdir(d):
            if f.endswith((".h", ".cuh")):
                m = max(m, os.path.getmtime(os.path.join(d, f)))
    return m


def _compile(unit: str, hdr_mtime: float, verbose: bool, bdir: str = BUILD, defs=()) -> str:
    src = os.path.join(CSRC, unit)
    obj = os.path.join(bdir, unit.replace(".cu", ".o"))
    if os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(src), hdr_mtime):
        return obj
    cmd = [nvcc(), *ARCH, *FLAGS, *EXTRA, *defs, "-c", src, "-o", obj]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {unit}:\n{r.stdout}\n{r.stderr}")
    if verbose:
        sys.stderr.write(r.stderr)
    return obj


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Compile every unit (parallel) and link liblqcd.so; returns its path.
    checked: the bounds-checked variant liblqcd_checked.so instead."""
    bdir, lib = (CHECKED_BUILD, CHECKED_LIB) if checked else (BUILD, LIB)
    defs = ("-DLQCD_CHECK_BOUNDS",) if checked else ()
    os.makedirs(bdir, exist_ok=True)
    if force:
        for f in os.listdir(bdir):
            if f.endswith(".o"):
                os.remove(os.path.join(bdir, f))
    hm = _headers_mtime()
    with ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        objs = list(ex.map(lambda u: _compile(u, hm, verbose, bdir, defs), UNITS))
    newest = max(os.path.getmtime(o) for o in objs)
    if not os.path.exists(lib) or os.path.getmtime(lib) < newest:
        tmp = f"{lib}.{os.getpid()}.tmp"
        cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart", "-lpthread"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
