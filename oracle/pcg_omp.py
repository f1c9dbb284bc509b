"""ctypes binding of ``pcg_omp.c``: the oracle's value update and FP64
Jacobi-PCG restated in plain C with OpenMP loops, for timing the oracle on
every host core.

TEST INFRASTRUCTURE ONLY, like ``repart_oracle``: the tests, the smoke check
and the CPU-baseline / reference legs of the benchmark use it; the product
path never does. Its inputs are the Python oracle's map (``PartMap``) and the
seeded inputs; its results are checked against ``repart_oracle.pcg`` in
``tests/test_oracle_pins.py``. ``build()`` compiles the library with the host
C compiler (no CUDA involved).
"""
from __future__ import annotations

import ctypes
import os
import shutil
import subprocess

import numpy as np

from . import repart_oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "pcg_omp.c")
LIB = os.path.join(HERE, "liborcpcg.so")


class _Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iterations", ctypes.c_int32),
                ("rel_residual", ctypes.c_double), ("true_rel_residual", ctypes.c_double)]


def build(force: bool = False) -> str:
    """Compile liborcpcg.so (OpenMP when the compiler has it, else serial)."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    cc = os.environ.get("CC") or shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        raise RuntimeError("no C compiler found for the oracle library")
    base = [cc, "-O2", "-std=c11", "-shared", "-fPIC", SRC, "-o", LIB, "-lm"]
    p = subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True, text=True)
    if p.returncode:
        p = subprocess.run(base, capture_output=True, text=True)
        if p.returncode:
            raise RuntimeError("oracle library build failed: " + p.stderr[-2000:])
    return LIB


_lib = None


def load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        i32, i64, dbl, vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
        lib.orc_threads.restype, lib.orc_threads.argtypes = ctypes.c_int, [ctypes.c_int]
        lib.orc_update_values.restype = None
        lib.orc_update_values.argtypes = [i64, vp, vp, vp, ctypes.c_int]
        lib.orc_jacobi_inverse.restype = None
        lib.orc_jacobi_inverse.argtypes = [i64, vp, vp, vp, ctypes.c_int]
        lib.orc_pcg.restype = ctypes.c_int
        lib.orc_pcg.argtypes = [i64, vp, vp, vp, vp, vp, dbl, i32, vp, ctypes.POINTER(_Result), ctypes.c_int]
        _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def threads(want: int = 0) -> int:
    """Threads a call with ``threads=want`` uses (0: every core OpenMP may use)."""
    return int(load().orc_threads(int(want)))


def update_values(src_of, buf, threads: int = 0) -> np.ndarray:
    """vals[p] = buf[src_of[p]] (Sec. 3, update procedure)."""
    src_of = np.ascontiguousarray(src_of, np.int32)
    buf = np.ascontiguousarray(buf, np.float64)
    vals = np.empty(src_of.shape[0], np.float64)
    load().orc_update_values(src_of.shape[0], _p(src_of), _p(buf), _p(vals), int(threads))
    return vals


def jacobi_inverse(diag_pos, vals, threads: int = 0) -> np.ndarray:
    diag_pos = np.ascontiguousarray(diag_pos, np.int32)
    vals = np.ascontiguousarray(vals, np.float64)
    dinv = np.empty(diag_pos.shape[0], np.float64)
    load().orc_jacobi_inverse(diag_pos.shape[0], _p(diag_pos), _p(vals), _p(dinv), int(threads))
    return dinv


def pcg(row_ptr, col_idx, vals, dinv, b, tol=1e-9, max_iter=10000, threads: int = 0) -> O.SolveResult:
    """Jacobi-PCG from x = 0, the steps of ``repart_oracle.pcg`` (same stopping
    test, true-residual confirmation and restart)."""
    row_ptr = np.ascontiguousarray(row_ptr, np.int32)
    col_idx = np.ascontiguousarray(col_idx, np.int32)
    vals = np.ascontiguousarray(vals, np.float64)
    dinv = np.ascontiguousarray(dinv, np.float64)
    b = np.ascontiguousarray(b, np.float64)
    n = b.shape[0]
    x = np.empty(n, np.float64)
    res = _Result()
    rc = load().orc_pcg(n, _p(row_ptr), _p(col_idx), _p(vals), _p(dinv), _p(b), float(tol), int(max_iter), _p(x),
                        ctypes.byref(res), int(threads))
    if rc:
        raise MemoryError("orc_pcg: host allocation failed")
    return O.SolveResult(x, res.iterations, res.status, res.rel_residual, res.true_rel_residual)
