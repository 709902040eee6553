"""Compiles libfpp.so in-tree for sm_103a with nvcc (no torch involvement).

Every translation unit is compiled in parallel, then linked with the CUDA
runtime statically.  The result is ``paper_2206_01382_gb300/_lib/libfpp.so``.
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
    if force or jobs or _newer(LIB, objs):
        cmd = [nvcc, ARCH, "-shared", "-o", LIB] + objs + ["-cudart", "static", "-lpthread"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            sys.stderr.write(r.stdout + r.stderr)
            raise RuntimeError("linking libfpp.so failed")
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
