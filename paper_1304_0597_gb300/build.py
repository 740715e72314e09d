"""Build libgame.so in-tree for sm_103a with nvcc (one translation unit per .cu, in parallel).

Usage: ``python -m paper_1304_0597_gb300.build`` (or ``__graft_entry__.build()``).
The library lands in ``paper_1304_0597_gb300/_lib/libgame.so``.  ``build(timeline=True)``
makes the profiling variant ``_lib/libgame_timeline.so`` (-DGAME_TC_TIMELINE: CTA 0 of the
tensor-core fitness kernel stamps its per-tile timeline; ``bench.py --timeline`` reads it).
"""

from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "libgame.so")
LIB_TIMELINE = os.path.join(OUT_DIR, "libgame_timeline.so")
LIB_CHECKS = os.path.join(OUT_DIR, "libgame_checks.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVFLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O3",
           "--expt-relaxed-constexpr", "-Xptxas", "-O3"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libgame.so")


def sources() -> list[str]:
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _compile(src: str, obj: str, extra: list[str]) -> str:
    cmd = [nvcc(), *ARCH, *NVFLAGS, *extra, "-I", CSRC, "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {os.path.basename(src)}:\n{r.stderr}")
    return r.stderr


def build(verbose: bool = False, extra: list[str] | None = None, timeline: bool = False,
          checks: bool = False) -> str:
    """Compile every csrc/*.cu and link libgame.so (or, with timeline, the profiling
    variant libgame_timeline.so; with checks, the bounds-checked debug variant
    libgame_checks.so built with -DGAME_CHECKS); returns the library path."""
    os.makedirs(OUT_DIR, exist_ok=True)
    extra = list(extra or []) + (["-DGAME_TC_TIMELINE"] if timeline else []) + \
        (["-DGAME_CHECKS"] if checks else [])
    lib = LIB_TIMELINE if timeline else LIB_CHECKS if checks else LIB
    objdir = os.path.join(OUT_DIR, "obj_timeline" if timeline else "obj_checks" if checks else "obj")
    os.makedirs(objdir, exist_ok=True)
    srcs = sources()
    objs = [os.path.join(objdir, os.path.basename(s)[:-3] + ".o") for s in srcs]
    with ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        logs = list(ex.map(lambda so: _compile(so[0], so[1], extra), zip(srcs, objs)))
    if verbose:
        for s, log in zip(srcs, logs):
            if log.strip():
                print(f"--- {os.path.basename(s)}\n{log}", file=sys.stderr)
    tmp = lib + ".tmp"
    cmd = [nvcc(), *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    v = "-v" in sys.argv
    extra = ["-Xptxas", "-v"] if "--ptxas-v" in sys.argv else None
    print(build(verbose=v or bool(extra), extra=extra))
