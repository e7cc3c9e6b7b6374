"""In-tree build of libdsasa.so (CUDA, sm_103a) with nvcc, and of libdsasa_peaks.so (the
arithmetic-roof microbenchmarks that bench.py reports beside the kernels).  build_checked()
makes the checked variant libdsasa_checked.so (-DDSASA_CHECKED: device bounds checks on the
atom kernels' data-dependent indices, reported as DSASA_ERR_CHECK), on demand only.

Each translation unit is compiled in parallel, then linked into the shared libraries with
the CUDA runtime linked statically.  No CMake, no torch extension machinery."""
from __future__ import annotations

import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libdsasa.so")
PEAKS_LIB = os.path.join(BUILD, "libdsasa_peaks.so")   # arithmetic-roof microbenchmarks (bench.py)
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE]
UNITS = ["dsasa_grid.cu", "dsasa_atoms_f32.cu", "dsasa_atoms_f64.cu", "dsasa_capi.cu", "dsasa_noalloc.cu", "dsasa_sr.cu"]
PEAK_UNITS = ["dsasa_peaks.cu"]
CHECKED_BUILD = os.path.join(BUILD, "checked")
CHECKED_LIB = os.path.join(CHECKED_BUILD, "libdsasa_checked.so")


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libdsasa.so")


def _deps():
    return glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        [os.path.join(INCLUDE, "dsasa.h"), __file__]


def up_to_date() -> bool:
    if not (os.path.exists(LIB) and os.path.exists(PEAKS_LIB)):
        return False
    t = min(os.path.getmtime(LIB), os.path.getmtime(PEAKS_LIB))
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force: bool = False, verbose: bool = False, extra_flags=()) -> str:
    """Compile libdsasa.so for sm_103a; returns its path."""
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    procs, objs, pobjs = [], [], []
    for u in UNITS + PEAK_UNITS:
        obj = os.path.join(BUILD, u.replace(".cu", ".o"))
        (pobjs if u in PEAK_UNITS else objs).append(obj)
        cmd = [cc, *ARCH, *FLAGS, *extra_flags, "-c", os.path.join(CSRC, u), "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        procs.append((u, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    errs = []
    for u, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            errs.append(f"--- {u}\n{out.decode(errors='replace')}")
        elif verbose and out:
            print(out.decode(errors="replace"))
    if errs:
        raise RuntimeError("nvcc failed:\n" + "\n".join(errs))
    for lib, o in ((LIB, objs), (PEAKS_LIB, pobjs)):
        tmp = lib + f".tmp{os.getpid()}"
        subprocess.check_call([cc, *ARCH, "-shared", "-o", tmp, *o])
        os.replace(tmp, lib)
    return LIB


def build_checked(force: bool = False) -> str:
    """Compile libdsasa_checked.so (the same sources with -DDSASA_CHECKED); returns its path."""
    if not force and os.path.exists(CHECKED_LIB) and \
            all(os.path.getmtime(d) <= os.path.getmtime(CHECKED_LIB) for d in _deps()):
        return CHECKED_LIB
    os.makedirs(CHECKED_BUILD, exist_ok=True)
    cc = nvcc()
    procs, objs = [], []
    for u in UNITS:
        obj = os.path.join(CHECKED_BUILD, u.replace(".cu", ".o"))
        objs.append(obj)
        cmd = [cc, *ARCH, *FLAGS, "-DDSASA_CHECKED", "-c", os.path.join(CSRC, u), "-o", obj]
        procs.append((u, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    errs = []
    for u, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            errs.append(f"--- {u}\n{out.decode(errors='replace')}")
    if errs:
        raise RuntimeError("nvcc failed:\n" + "\n".join(errs))
    tmp = CHECKED_LIB + f".tmp{os.getpid()}"
    subprocess.check_call([cc, *ARCH, "-shared", "-o", tmp, *objs])
    os.replace(tmp, CHECKED_LIB)
    return CHECKED_LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True))
