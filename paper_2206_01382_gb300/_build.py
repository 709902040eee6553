"""Compiles libfpp.so in-tree for sm_103a with nvcc (no torch involvement).

Every translation unit is compiled in parallel, then linked with the CUDA
runtime statically.  The result is ``paper_2206_01382_gb300/_lib/libfpp.so``,
and beside it ``libfpp_debug.so``: the same library with the search kernels
compiled with FPP_DEBUG_BOUNDS (device checks of every gather and scatter
index of the candidate path, in place of a memory checker).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
OUT = os.path.join(PKG, "_lib")
LIB = os.path.join(OUT, "libfpp.so")
LIB_DEBUG = os.path.join(OUT, "libfpp_debug.so")
DEBUG_UNITS = ("search_kernels.cu",)   # compiled a second time with FPP_DEBUG_BOUNDS
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found")
    return p


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC)
                  if f.endswith((".cu", ".cpp")))


def _newer(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False, force: bool = False, extra: list | None = None) -> str:
    os.makedirs(OUT, exist_ok=True)
    nvcc = _nvcc()
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    headers.append(os.path.join(os.path.dirname(PKG), "include", "fpp.h"))
    common = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-lineinfo",
              "-I" + os.path.join(os.path.dirname(PKG), "include")] + (extra or [])
    jobs = []
    for src in sources():
        obj = os.path.join(OUT, os.path.basename(src) + ".o")
        if force or _newer(obj, [src] + headers):
            if src.endswith(".cu"):
                cmd = [nvcc, ARCH, "-c", src, "-o", obj, "--expt-relaxed-constexpr",
                       "-Xptxas", "-warn-spills"] + common
            else:
                cmd = [nvcc, "-x", "c++", "-c", src, "-o", obj] + common
            jobs.append((src, cmd))
        if os.path.basename(src) in DEBUG_UNITS:
            dobj = os.path.join(OUT, os.path.basename(src) + ".debug.o")
            if force or _newer(dobj, [src] + headers):
                jobs.append((src, [nvcc, ARCH, "-c", src, "-o", dobj, "--expt-relaxed-constexpr",
                                   "-DFPP_DEBUG_BOUNDS"] + common))
    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 4)) as ex:
        futs = {ex.submit(subprocess.run, cmd, capture_output=True, text=True): src
                for src, cmd in jobs}
        for f in cf.as_completed(futs):
            r = f.result()
            if verbose or r.returncode != 0:
                sys.stderr.write(r.stdout + r.stderr)
            if r.returncode != 0:
                raise RuntimeError(f"compiling {futs[f]} failed")
    objs = [os.path.join(OUT, os.path.basename(s) + ".o") for s in sources()]
    dobjs = [os.path.join(OUT, os.path.basename(s) + (".debug.o" if os.path.basename(s) in DEBUG_UNITS
                                                      else ".o")) for s in sources()]
    for lib, ob in ((LIB, objs), (LIB_DEBUG, dobjs)):
        if force or jobs or _newer(lib, ob):
            cmd = [nvcc, ARCH, "-shared", "-o", lib] + ob + ["-cudart", "static", "-lpthread"]
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                sys.stderr.write(r.stdout + r.stderr)
                raise RuntimeError(f"linking {os.path.basename(lib)} failed")
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
