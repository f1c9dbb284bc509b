"""Build librepart.so in-tree with nvcc for sm_103a (GB300).

Each translation unit compiles in parallel into ``_build/``; the shared
library lands next to this file, where the binding loads it from. The
bounds-checked variant (``check=True``: every device gather index and derived
offset range-checked, violations counted instead of trapping, see
rp_check_violations) compiles the same sources with -DRP_CHECK into
``_build_check/`` and ``librepart_check.so``.
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
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "librepart.so")
BUILD_CHECK = os.path.join(HERE, "_build_check")
LIB_CHECK = os.path.join(HERE, "librepart_check.so")
SOURCES = ["rp_map.cu", "rp_update.cu", "rp_pcg.cu", "rp_adjoint.cu", "rp_batch.cu", "rp_noalloc.cu", "rp_sliced.cu", "rp_bicgstab.cu"]
HEADERS = [os.path.join(CSRC, h) for h in sorted(os.listdir(CSRC)) if h.endswith(".cuh")] + [
    os.path.join(ROOT, "include", "repart.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include")]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build librepart")


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _run(cmd, verbose):
    p = subprocess.run(cmd, capture_output=True, text=True)
    if verbose or p.returncode:
        sys.stderr.write(" ".join(cmd) + "\n" + p.stdout + p.stderr)
    if p.returncode:
        raise RuntimeError(f"nvcc failed on {cmd[-3]}")


def build(force: bool = False, verbose: bool = False, extra_flags=(), check: bool = False,
          with_check: bool = False) -> str:
    """Compile the library (check: the bounds-checked variant instead;
    with_check: both, their units compiled together). Returns the path of the
    library asked for (the normal one when with_check)."""
    cc = nvcc()
    variants = [(BUILD_CHECK, LIB_CHECK, ["-DRP_CHECK"])] if check else [(BUILD, LIB, [])]
    if with_check and not check:
        variants.append((BUILD_CHECK, LIB_CHECK, ["-DRP_CHECK"]))
    jobs, links = [], []
    for bdir, lib, defs in variants:
        os.makedirs(bdir, exist_ok=True)
        objs, n0 = [], len(jobs)
        for src in SOURCES:
            s = os.path.join(CSRC, src)
            o = os.path.join(bdir, src.replace(".cu", ".o"))
            objs.append(o)
            if force or _stale(o, [s] + HEADERS):
                jobs.append([cc, *ARCH, *FLAGS, *defs, *extra_flags, "-c", s, "-o", o])
        if force or len(jobs) > n0 or _stale(lib, objs):
            links.append([cc, *ARCH, "-shared", "-o", lib, *objs, "-cudart", "static", "-lcuda"])
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 1))) as ex:
        list(ex.map(lambda c: _run(c, verbose), jobs))
    for cmd in links:
        _run(cmd, verbose)
    return variants[0][1]


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
