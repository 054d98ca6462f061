"""In-tree build of libsfchem.so (nvcc, sm_103a only).

The translation units are compiled in parallel and linked into one
shared library next to this file.  Rebuilds only when a source is newer than
the library.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OBJ = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libsfchem.so")
BENCH_LIB = os.path.join(HERE, "libsfbench.so")
UNITS = ("li_fp64.cu", "li_mixed.cu", "li_mixed_ff.cu", "li_mixed_masked.cu", "nr_fp64.cu", "sfchem_abi.cu",
         "noalloc.cu", "photon.cu", "derived.cu")
BENCH_UNITS = ("microbench.cu",)
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", CSRC, "-I", INCLUDE]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: libsfchem needs the CUDA toolkit to build")


def _sources():
    out = [os.path.join(CSRC, f) for f in os.listdir(CSRC)
           if f.endswith((".cu", ".cuh", ".h")) and f not in BENCH_UNITS]
    out.append(os.path.join(INCLUDE, "sfchem.h"))
    return out


def stale() -> bool:
    # the benchmark library also includes the solver's device header
    bench_srcs = [os.path.join(CSRC, u) for u in BENCH_UNITS] + [os.path.join(CSRC, "li_device.cuh")]
    for lib, srcs in ((LIB, _sources()), (BENCH_LIB, bench_srcs)):
        if not os.path.exists(lib):
            return True
        t = os.path.getmtime(lib)
        if any(os.path.getmtime(p) > t for p in srcs):
            return True
    return False


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not stale():
        return LIB
    nvcc = _nvcc()
    os.makedirs(OBJ, exist_ok=True)

    def compile_one(u):
        obj = os.path.join(OBJ, u.replace(".cu", ".o"))
        cmd = [nvcc, *ARCH, *FLAGS, "-c", os.path.join(CSRC, u), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {u}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(len(UNITS) + len(BENCH_UNITS)) as ex:
        objs = list(ex.map(compile_one, UNITS + BENCH_UNITS))
    for lib, part in ((LIB, objs[:len(UNITS)]), (BENCH_LIB, objs[len(UNITS):])):
        tmp = lib + ".tmp"
        cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *part]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
