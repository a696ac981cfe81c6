"""Build the CUDA library ``_lib/libmg.so`` in-tree for sm_103a.

Each translation unit is compiled by its own ``nvcc`` process (in parallel),
then linked into one shared library with the CUDA runtime linked statically.
Beside it, ``_lib/libmg_checked.so`` is the bounds-checked variant of the same
sources (``-DMG_CHECKED``: every device index taken from a host table is
checked before use; grid sizes n <= 32 only, so it compiles quickly); the
binding loads it instead of the main library when MG_CHECKED=1 is set.
Run as ``python -m paper_1402_1763_gb300.build`` or call ``build()``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "libmg.so")
LIB_CHECKED = os.path.join(OUT_DIR, "libmg_checked.so")
CHECKED_FLAGS = ["-DMG_CHECKED", "-DMG_MAX_N=32"]
SOURCES = ["mg_pass_yz_f32.cu", "mg_pass_yz_f64.cu", "mg_pass_x.cu", "mg_api.cu", "mg_noalloc.cu", "mg_persist.cu", "mg_peak.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def nvcc_path() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _stale(out: str, deps) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False, force: bool = False) -> str:
    """Compile (where stale) and link both libraries; returns the main one's path."""
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = nvcc_path()
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    headers.append(os.path.join(os.path.dirname(HERE), "include", "mg.h"))
    variants = [(LIB, "", []), (LIB_CHECKED, "_checked", CHECKED_FLAGS)]
    objs = {lib: [] for lib, _, _ in variants}
    jobs = []
    for lib, suffix, extra in variants:
        for src in SOURCES:
            s = os.path.join(CSRC, src)
            o = os.path.join(OUT_DIR, src.replace(".cu", suffix + ".o"))
            objs[lib].append(o)
            if force or _stale(o, [s] + headers):
                jobs.append([nvcc] + ARCH + FLAGS + extra + ["-c", s, "-o", o])
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            futs = [ex.submit(subprocess.run, j, capture_output=True, text=True) for j in jobs]
            for j, f in zip(jobs, futs):
                r = f.result()
                if verbose or r.returncode != 0:
                    sys.stderr.write(r.stdout + r.stderr)
                if r.returncode != 0:
                    raise RuntimeError("nvcc failed: " + " ".join(j))
    for lib, _, _ in variants:
        if force or jobs or _stale(lib, objs[lib]):
            cmd = [nvcc] + ARCH + ["-shared", "-cudart", "static", "-o", lib] + objs[lib]
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                sys.stderr.write(r.stdout + r.stderr)
                raise RuntimeError("link failed: " + lib)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
