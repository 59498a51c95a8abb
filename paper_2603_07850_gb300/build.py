"""Build libgoldbach_gb300.so in-tree with nvcc for sm_103a (GB300).

Translation units are compiled in parallel and linked with the static CUDA
runtime, so the library loads without torch and without a runtime search path.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libgoldbach_gb300.so")
# the same library with per-phase cycle counters in the kernels (GB_PHASE_CLOCKS)
PHASES_OUT_DIR = os.path.join(HERE, "_build_phases")
PHASES_LIB = os.path.join(HERE, "libgoldbach_gb300_phases.so")
# the same library with bounds checks on the shared-memory window (GB_DEBUG)
DEBUG_OUT_DIR = os.path.join(HERE, "_build_debug")
DEBUG_LIB = os.path.join(HERE, "libgoldbach_gb300_debug.so")
SOURCES = ["gb_kernels.cu", "gb_persist_256.cu", "gb_persist_512.cu", "gb_persist_768.cu", "gb_persist_1024.cu",
           "gb_pipe_8.cu",
           "gb_pipe_16.cu",
           "gb_capi.cu", "gb_serve.cpp", "gb_noalloc.cu", "gb_peaks.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _flags(src: str, phases: bool = False, debug: bool = False) -> list[str]:
    f = ["-std=c++17", "-O3", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include")]
    if phases:
        f.append("-DGB_PHASE_CLOCKS")
    if debug:
        f.append("-DGB_DEBUG")
    if src.endswith(".cu"):
        f += ARCH + ["-lineinfo", "--expt-relaxed-constexpr"]
    else:
        f += ["-x", "cu"] + ARCH
    return f


def _stale(out: str, deps: list[str]) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, phases: bool = False, debug: bool = False) -> str:
    """Build the library and return its path.  phases=True builds the variant
    with per-phase cycle counters, debug=True the variant with bounds checks
    on every shared-memory window access; each is a separate file."""
    if phases and debug:
        raise ValueError("one variant at a time")
    out_dir, lib = ((PHASES_OUT_DIR, PHASES_LIB) if phases else (DEBUG_OUT_DIR, DEBUG_LIB) if debug
                    else (OUT_DIR, LIB))
    os.makedirs(out_dir, exist_ok=True)
    headers = [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith((".h", ".cuh"))]
    headers.append(os.path.join(ROOT, "include", "goldbach_gb300.h"))
    objs = []
    jobs = []
    for s in SOURCES:
        src = os.path.join(CSRC, s)
        obj = os.path.join(out_dir, s + ".o")
        objs.append(obj)
        if force or _stale(obj, [src] + headers + [__file__]):
            cmd = [nvcc()] + _flags(s, phases, debug) + ["-c", src, "-o", obj]
            jobs.append(cmd)
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        for cmd, res in zip(jobs, ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), jobs)):
            if verbose or res.returncode:
                sys.stderr.write(" ".join(cmd) + "\n" + res.stdout + res.stderr)
            if res.returncode:
                raise RuntimeError(f"nvcc failed: {' '.join(cmd)}")
    if force or jobs or _stale(lib, objs):
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [nvcc()] + ARCH + ["-shared", "-cudart", "static", "-o", tmp] + objs
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode:
            sys.stderr.write(" ".join(cmd) + "\n" + res.stdout + res.stderr)
            raise RuntimeError("link failed")
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
