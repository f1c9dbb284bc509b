"""Python binding of librepart (argument marshalling only).

Every function here has the name of the C-ABI call it wraps (without the
``rp_`` prefix) and only converts arguments: NumPy arrays for the host
descriptors, torch tensors (device or host) for the value and vector
buffers, the current torch stream as the CUDA stream. All computation runs
in the library's CUDA kernels. There is no fallback: if the library is
missing, loading fails with an error.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librepart.so")

RP_OK, RP_EINVAL, RP_EDUP, RP_ERANGE, RP_EOVERFLOW, RP_ENOMEM, RP_ECUDA = range(7)
RP_NOT_CONVERGED, RP_BREAKDOWN, RP_DEVICE_TIMEOUT, RP_EUNSUPPORTED = 7, 8, 9, 10
RP_MEM_DEVICE, RP_MEM_HOST, RP_MEM_HOST_DIRECT, RP_MEM_HOST_ASYNC = 0, 1, 2, 3
RP_FP64, RP_MIXED, RP_MIXED_RU = 0, 1, 2
RP_LAYOUT_AUTO, RP_LAYOUT_CSR = 0, 1
RP_PRECOND_JACOBI, RP_PRECOND_LINE = 0, 1
PRECISIONS = {"fp64": RP_FP64, "mixed": RP_MIXED, "mixed_ru": RP_MIXED_RU}

_i32p = ctypes.POINTER(ctypes.c_int32)


class LduDesc(ctypes.Structure):
    _fields_ = [("n_cells", ctypes.c_int32), ("n_faces", ctypes.c_int32),
                ("lower_addr", _i32p), ("upper_addr", _i32p),
                ("n_iface", ctypes.c_int32), ("iface_row", _i32p),
                ("iface_nbr_rank", _i32p), ("iface_nbr_col", _i32p)]


class Options(ctypes.Structure):
    _fields_ = [("n_parts", ctypes.c_int32), ("symmetric", ctypes.c_int32),
                ("want_fp32", ctypes.c_int32), ("want_transpose", ctypes.c_int32),
                ("max_iter", ctypes.c_int32), ("max_outer", ctypes.c_int32),
                ("max_restarts", ctypes.c_int32), ("device", ctypes.c_int32),
                ("inner_tol", ctypes.c_double), ("spin_limit", ctypes.c_int64),
                ("host_loop", ctypes.c_int32), ("layout", ctypes.c_int32), ("ru_delta", ctypes.c_double),
                ("precond", ctypes.c_int32), ("spare", ctypes.c_int32)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iterations", ctypes.c_int32),
                ("outer_iterations", ctypes.c_int32), ("restarts", ctypes.c_int32), ("passes", ctypes.c_int32),
                ("rel_residual", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class SlicedView(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in ("n_slices", "n_entries", "ibuf_len", "tabs_len")] + \
               [(k, ctypes.c_void_p) for k in ("desc", "tinfo", "tabs", "ibuf", "pos", "vals", "vals32", "srow",
                                               "vals32s", "scale")] + [("uniform4", ctypes.c_int32)]


class MapView(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in ("n_rows", "nnz", "nl_nnz", "n_nl_cols", "row_off", "buf_off", "buf_len")] + \
               [(k, ctypes.c_void_p) for k in ("row_ptr", "col_idx", "src_of", "diag_pos", "tpos", "nl_row_ptr",
                                               "nl_col_idx", "nl_src_of", "nl_cols")]


_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load librepart.so (built by ``build.build()``); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"librepart.so not found at {path}: build it with paper_2510_08536_gb300.build.build()")
    lib = ctypes.CDLL(path)
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    sig = {
        "rp_default_options": (None, [ctypes.POINTER(Options)]),
        "rp_build_repartition": (i32, [ctypes.POINTER(LduDesc), i32, ctypes.POINTER(Options), ctypes.POINTER(vp)]),
        "rp_get_part_map": (i32, [vp, i32, ctypes.POINTER(MapView)]),
        "rp_get_sizes": (i32, [vp, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i32)]),
        "rp_update_values_packed": (i32, [vp, vp, i32, vp]),
        "rp_update_values": (i32, [vp, vp, vp, vp, vp, i32, vp]),
        "rp_get_values": (i32, [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp)]),
        "rp_spmv": (i32, [vp, vp, vp, vp, vp]),
        "rp_iter_spmv": (i32, [vp, vp, vp, i32, vp]),
        "rp_get_sliced_view": (i32, [vp, ctypes.POINTER(SlicedView)]),
        "rp_spmv_noalloc": (i32, [i64, vp, vp, vp, vp, vp, vp, vp]),
        "rp_batch_build": (i32, [ctypes.POINTER(LduDesc), i32, ctypes.POINTER(Options), ctypes.POINTER(vp)]),
        "rp_batch_update_solve": (i32, [vp, vp, i32, vp, vp, dbl, i32, ctypes.POINTER(SolveInfo), vp]),
        "rp_batch_set_config": (i32, [vp, i32, i32]),
        "rp_set_solver_options": (i32, [vp, ctypes.POINTER(Options)]),
        "rp_batch_autotune": (i32, [vp, vp, vp, vp, dbl, i32, ctypes.POINTER(i32), ctypes.POINTER(i32),
                                    ctypes.POINTER(ctypes.c_float), vp]),
        "rp_solve": (i32, [vp, vp, vp, dbl, i32, i32, i32, ctypes.POINTER(SolveInfo), vp]),
        "rp_get_solve_info": (i32, [vp, ctypes.POINTER(SolveInfo), vp]),
        "rp_solve_bicgstab": (i32, [vp, vp, vp, dbl, i32, i32, ctypes.POINTER(SolveInfo), vp]),
        "rp_solve_bicgstab_mixed": (i32, [vp, vp, vp, dbl, i32, i32, ctypes.POINTER(SolveInfo), vp]),
        "rp_solve_adjoint": (i32, [vp, vp, vp, dbl, ctypes.POINTER(SolveInfo), vp]),
        "rp_profile_iteration": (i32, [vp, vp, i32, i32, ctypes.POINTER(ctypes.c_float), vp]),
        "rp_entry_grad": (i32, [vp, vp, vp, vp, vp]),
        "rp_face_grad": (i32, [vp, vp, vp, vp, vp]),
        "rp_check_violations": (i32, [ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(i32), ctypes.POINTER(i64), i32]),
        "rp_destroy": (None, [vp]),
        "rp_status_str": (ctypes.c_char_p, [i32]),
        "rp_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


class RepartError(RuntimeError):
    def __init__(self, status: int, where: str):
        lib = load()
        self.status = status
        super().__init__(f"{where}: {lib.rp_status_str(status).decode()} - {lib.rp_last_error().decode()}")


def _check(status: int, where: str, ok=(RP_OK,)):
    if status not in ok:
        raise RepartError(status, where)
    return status


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _ptr(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _where(t) -> int:
    return RP_MEM_DEVICE if t.is_cuda else RP_MEM_HOST


def _f64(t, name):
    import torch
    if t.dtype != torch.float64 or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous float64 tensor")
    return t


class Handle:
    """Owns one rp_handle; destroyed with the object."""

    def __init__(self, ptr: int, symmetric: bool):
        self.ptr = ctypes.c_void_p(ptr)
        self.symmetric = symmetric
        n, nnz, slots, parts = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
        _check(load().rp_get_sizes(self.ptr, n, nnz, slots, parts), "rp_get_sizes")
        self.n, self.nnz, self.n_slots, self.n_parts = n.value, nnz.value, slots.value, parts.value

    def close(self):
        if self.ptr:
            load().rp_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def default_options() -> Options:
    o = Options()
    load().rp_default_options(ctypes.byref(o))
    return o


def build_repartition(ranks, n_parts: int = 1, symmetric: bool = False, want_fp32: bool = True,
                      want_transpose: bool = False, **opts) -> Handle:
    """rp_build_repartition over objects with the rp_ldu_desc fields (NumPy arrays)."""
    lib = load()
    k = len(ranks)
    descs = (LduDesc * k)()
    keep = []
    for i, r in enumerate(ranks):
        arrs = [np.ascontiguousarray(getattr(r, f), dtype=np.int32) for f in
                ("lower_addr", "upper_addr", "iface_row", "iface_nbr_rank", "iface_nbr_col")]
        keep.append(arrs)
        p = [a.ctypes.data_as(_i32p) for a in arrs]
        descs[i] = LduDesc(int(r.n_cells), arrs[0].shape[0], p[0], p[1], arrs[2].shape[0], p[2], p[3], p[4])
    o = default_options()
    o.n_parts, o.symmetric, o.want_fp32, o.want_transpose = n_parts, int(symmetric), int(want_fp32), int(want_transpose)
    for key, val in opts.items():
        setattr(o, key, val)
    out = ctypes.c_void_p()
    _check(lib.rp_build_repartition(descs, k, ctypes.byref(o), ctypes.byref(out)), "rp_build_repartition")
    h = Handle(out.value, symmetric)
    h.options = o
    return h


class _CudaArray:
    """Non-owning __cuda_array_interface__ view of a handle-owned buffer."""

    def __init__(self, ptr, n, typestr):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": typestr, "data": (int(ptr or 0), False),
                                         "version": 3, "strides": None}


def _view(ptr, n, typestr):
    import torch
    if n == 0 or not ptr:
        dt = {"<i4": torch.int32, "<f8": torch.float64, "<f4": torch.float32}[typestr]
        return torch.zeros(0, dtype=dt, device="cuda")
    return torch.as_tensor(_CudaArray(ptr, n, typestr), device="cuda")


def get_part_map(h: Handle, part: int = 0) -> dict:
    """rp_get_part_map, copied into torch tensors on the device."""
    v = MapView()
    _check(load().rp_get_part_map(h.ptr, part, ctypes.byref(v)), "rp_get_part_map")
    import torch
    torch.cuda.synchronize()
    out = dict(n_rows=v.n_rows, nnz=v.nnz, nl_nnz=v.nl_nnz, n_nl_cols=v.n_nl_cols, row_off=v.row_off,
               buf_off=v.buf_off, buf_len=v.buf_len)
    sizes = dict(row_ptr=v.n_rows + 1, col_idx=v.nnz, src_of=v.nnz, diag_pos=v.n_rows, tpos=v.nnz,
                 nl_row_ptr=v.n_rows + 1, nl_col_idx=v.nl_nnz, nl_src_of=v.nl_nnz, nl_cols=v.n_nl_cols)
    for key, cnt in sizes.items():
        ptr = getattr(v, key)
        out[key] = None if (key == "tpos" and not ptr) else _view(ptr, cnt, "<i4").clone()
    return out


def get_values(h: Handle) -> dict:
    """rp_get_values as non-owning device views (valid until the next update)."""
    vals, vals32, dinv = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
    _check(load().rp_get_values(h.ptr, ctypes.byref(vals), ctypes.byref(vals32), ctypes.byref(dinv)), "rp_get_values")
    return dict(vals=_view(vals.value, h.nnz, "<f8"),
                vals32=_view(vals32.value, h.nnz, "<f4") if vals32.value else None,
                dinv=_view(dinv.value, h.n, "<f8"))


def update_values_packed(h: Handle, buffer, stream=None, direct: bool = False, asynchronous: bool = False):
    """rp_update_values_packed; a host buffer is copied to the device first (on
    the handle's own copy stream, overlapping earlier work, when
    ``asynchronous``), or read in place by the permutation kernel when ``direct``."""
    _f64(buffer, "buffer")
    if buffer.numel() != h.n_slots:
        raise ValueError(f"buffer has {buffer.numel()} values, the handle needs {h.n_slots}")
    if direct and asynchronous:
        raise ValueError("direct and asynchronous exclude each other")
    where = _where(buffer)
    if not buffer.is_cuda and direct:
        where = RP_MEM_HOST_DIRECT
    elif not buffer.is_cuda and asynchronous:
        where = RP_MEM_HOST_ASYNC
    _check(load().rp_update_values_packed(h.ptr, _ptr(buffer), where, _stream(stream)), "rp_update_values_packed")


def update_values(h: Handle, diag, upper, lower, iface, stream=None):
    """Per-rank lists of float64 tensors, all on the host or all on the device."""
    k = len(diag)
    arr = lambda ts: (ctypes.c_void_p * k)(*[0 if t is None else t.data_ptr() for t in ts])
    where = _where(diag[0])
    lo = arr(lower) if lower is not None else None
    _check(load().rp_update_values(h.ptr, arr(diag), arr(upper), lo, arr(iface), where, _stream(stream)),
           "rp_update_values")


def spmv(h: Handle, x, y, xy=None, stream=None):
    _check(load().rp_spmv(h.ptr, _ptr(x), _ptr(y), _ptr(xy), _stream(stream)), "rp_spmv")


def iter_spmv(h: Handle, x, y, precision: str = "fp64", stream=None):
    """rp_iter_spmv: y = A x with the PCG iteration's own kernel (float64 x/y
    for "fp64", float32 x/y on the FP32 values otherwise)."""
    _check(load().rp_iter_spmv(h.ptr, _ptr(x), _ptr(y), PRECISIONS[precision], _stream(stream)), "rp_iter_spmv")


def sliced_sizes(h: Handle):
    """(n_slices, n_entries, ibuf_len, tabs_len) of the sliced layout, or None
    when the iteration runs on the CSR arrays."""
    v = SlicedView()
    _check(load().rp_get_sliced_view(h.ptr, ctypes.byref(v)), "rp_get_sliced_view")
    return (v.n_slices, v.n_entries, v.ibuf_len, v.tabs_len) if v.n_slices else None


def sliced_uniform4(h: Handle) -> bool:
    """Whether every slice has 4-bit indices and rows of at most 8 entries (the
    iteration then runs the uniform-slice instance of its SpMV kernel)."""
    v = SlicedView()
    _check(load().rp_get_sliced_view(h.ptr, ctypes.byref(v)), "rp_get_sliced_view")
    return bool(v.n_slices and v.uniform4)


def inner_scaled(h: Handle) -> bool:
    """Whether the mixed solves' FP32 iteration runs on the scaled system S A S
    (made by the first mixed solve on a handle that takes it)."""
    v = SlicedView()
    _check(load().rp_get_sliced_view(h.ptr, ctypes.byref(v)), "rp_get_sliced_view")
    return bool(v.vals32s)


def get_sliced_view(h: Handle) -> dict:
    """rp_get_sliced_view, copied into torch tensors on the device (None when
    the iteration runs on the CSR arrays)."""
    v = SlicedView()
    _check(load().rp_get_sliced_view(h.ptr, ctypes.byref(v)), "rp_get_sliced_view")
    if v.n_slices == 0:
        return None
    import torch
    torch.cuda.synchronize()
    return dict(n_slices=v.n_slices, n_entries=v.n_entries, ibuf_len=v.ibuf_len, tabs_len=v.tabs_len,
                desc=_view(v.desc, 2 * (v.n_slices + 1), "<i4").clone(),
                tinfo=_view(v.tinfo, v.n_slices, "<i4").clone(),
                tabs=_view(v.tabs, v.tabs_len, "<i4").clone(),
                ibuf=_view(v.ibuf, v.ibuf_len, "<i4").clone(),
                pos=_view(v.pos, v.n_entries, "<i4").clone(),
                vals=_view(v.vals, v.n_entries, "<f8").clone(),
                vals32=_view(v.vals32, v.n_entries, "<f4").clone() if v.vals32 else None,
                srow=_view(v.srow, 2 * v.n_slices, "<i4").clone() if v.srow else None,
                vals32s=_view(v.vals32s, v.n_entries, "<f4").clone() if v.vals32s else None,
                scale=_view(v.scale, h.n, "<f8").clone() if v.scale else None, uniform4=bool(v.uniform4))


def batch_build(systems, want_fp32: bool = True, **opts) -> Handle:
    """rp_batch_build: one handle holding every independent system (one part each)."""
    lib = load()
    k = len(systems)
    descs = (LduDesc * k)()
    keep = []
    for i, r in enumerate(systems):
        lo = np.ascontiguousarray(r.lower_addr, dtype=np.int32)
        up = np.ascontiguousarray(r.upper_addr, dtype=np.int32)
        keep.append((lo, up))
        descs[i] = LduDesc(int(r.n_cells), lo.shape[0], lo.ctypes.data_as(_i32p), up.ctypes.data_as(_i32p), 0,
                           None, None, None)
    o = default_options()
    o.want_fp32 = int(want_fp32)
    for key, val in opts.items():
        setattr(o, key, val)
    out = ctypes.c_void_p()
    _check(lib.rp_batch_build(descs, k, ctypes.byref(o), ctypes.byref(out)), "rp_batch_build")
    h = Handle(out.value, False)
    h.options = o
    return h


def batch_update_solve(h: Handle, buffer, b, x, tol: float = 1e-9, precision: str = "fp64", stream=None,
                       wait: bool = True):
    """rp_batch_update_solve; returns per-system SolveInfo dicts when ``wait``."""
    _f64(buffer, "buffer"); _f64(b, "b"); _f64(x, "x")
    prec = PRECISIONS[precision]
    infos = (SolveInfo * h.n_parts)() if wait else None
    st = load().rp_batch_update_solve(h.ptr, _ptr(buffer), _where(buffer), _ptr(b), _ptr(x), float(tol), prec,
                                      infos, _stream(stream))
    _check(st, "rp_batch_update_solve", ok=(RP_OK, RP_NOT_CONVERGED, RP_BREAKDOWN))
    return [i.as_dict() for i in infos] if wait else None


def set_solver_options(h: Handle, **kw):
    """rp_set_solver_options: change max_iter / max_outer / max_restarts /
    inner_tol / ru_delta / host_loop / precond / spin_limit of an existing handle."""
    o = h.options if getattr(h, "options", None) is not None else default_options()
    for key, val in kw.items():
        setattr(o, key, val)
    _check(load().rp_set_solver_options(h.ptr, ctypes.byref(o)), "rp_set_solver_options")
    h.options = o


def batch_set_config(h: Handle, cluster: int, threads: int):
    _check(load().rp_batch_set_config(h.ptr, int(cluster), int(threads)), "rp_batch_set_config")


def batch_autotune(h: Handle, buffer, b, x, tol: float = 1e-9, precision: str = "fp64", stream=None):
    """rp_batch_autotune: returns (cluster, threads, ms) of the fastest launch shape."""
    c, t, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_float()
    prec = PRECISIONS[precision]
    _check(load().rp_batch_autotune(h.ptr, _ptr(buffer), _ptr(b), _ptr(x), float(tol), prec, ctypes.byref(c),
                                    ctypes.byref(t), ctypes.byref(ms), _stream(stream)), "rp_batch_autotune")
    return c.value, t.value, ms.value


def spmv_noalloc(n: int, row_ptr, col_idx, vals, x, y, xy=None, stream=None):
    """rp_spmv_noalloc: the same product for a caller-owned CSR matrix, with no
    device allocation (for callers that cannot allocate device memory)."""
    _check(load().rp_spmv_noalloc(int(n), _ptr(row_ptr), _ptr(col_idx), _ptr(vals), _ptr(x), _ptr(y), _ptr(xy),
                                  _stream(stream)), "rp_spmv_noalloc")


def solve(h: Handle, b, x, tol: float = 1e-9, precision: str = "fp64", x_is_guess: bool = False,
          stream=None, wait: bool = True, raise_on_status: bool = False):
    """rp_solve; returns the SolveInfo as a dict when ``wait`` (else None)."""
    _f64(b, "b"); _f64(x, "x")
    if b.is_cuda != x.is_cuda:
        raise ValueError("b and x must both live on the device or both on the host")
    prec = PRECISIONS[precision]
    info = SolveInfo()
    st = load().rp_solve(h.ptr, _ptr(b), _ptr(x), float(tol), prec, int(x_is_guess), _where(b),
                         ctypes.byref(info) if wait else None, _stream(stream))
    _check(st, "rp_solve", ok=(RP_OK,) if raise_on_status else (RP_OK, RP_NOT_CONVERGED, RP_BREAKDOWN))
    return info.as_dict() if wait else None


def solve_info(h: Handle, stream=None) -> dict:
    """rp_get_solve_info: waits for the stream and returns the SolveInfo of the
    latest solve launched with ``wait=False``."""
    info = SolveInfo()
    st = load().rp_get_solve_info(h.ptr, ctypes.byref(info), _stream(stream))
    _check(st, "rp_get_solve_info", ok=(RP_OK, RP_NOT_CONVERGED, RP_BREAKDOWN))
    return info.as_dict()


def solve_bicgstab(h: Handle, b, x, tol: float = 1e-9, x_is_guess: bool = False, stream=None,
                   wait: bool = True, raise_on_status: bool = False, precision: str = "fp64"):
    """rp_solve_bicgstab (non-symmetric systems; precision "fp64") or
    rp_solve_bicgstab_mixed ("mixed": FP32 inner solves in FP64 refinement);
    returns the SolveInfo as a dict when ``wait``."""
    _f64(b, "b"); _f64(x, "x")
    if b.is_cuda != x.is_cuda:
        raise ValueError("b and x must both live on the device or both on the host")
    if precision not in ("fp64", "mixed"):
        raise ValueError("precision must be 'fp64' or 'mixed'")
    name = "rp_solve_bicgstab" if precision == "fp64" else "rp_solve_bicgstab_mixed"
    info = SolveInfo()
    st = getattr(load(), name)(h.ptr, _ptr(b), _ptr(x), float(tol), int(x_is_guess), _where(b),
                               ctypes.byref(info) if wait else None, _stream(stream))
    _check(st, name, ok=(RP_OK,) if raise_on_status else (RP_OK, RP_NOT_CONVERGED, RP_BREAKDOWN))
    return info.as_dict() if wait else None


def profile_iteration(h: Handle, b, precision: str = "fp64", iters: int = 20, stream=None):
    """rp_profile_iteration: average ms of the SpMV, residual and x/p kernels."""
    ms = (ctypes.c_float * 3)()
    prec = PRECISIONS[precision]
    _check(load().rp_profile_iteration(h.ptr, _ptr(b), prec, int(iters), ms, _stream(stream)), "rp_profile_iteration")
    return dict(spmv=ms[0], resid=ms[1], xp=ms[2])


def solve_adjoint(h: Handle, g, lam, tol: float = 1e-9, stream=None, wait: bool = True):
    info = SolveInfo()
    st = load().rp_solve_adjoint(h.ptr, _ptr(g), _ptr(lam), float(tol), ctypes.byref(info) if wait else None,
                                 _stream(stream))
    _check(st, "rp_solve_adjoint", ok=(RP_OK, RP_NOT_CONVERGED, RP_BREAKDOWN))
    return info.as_dict() if wait else None


def entry_grad(h: Handle, lam, x, g_buffer, stream=None):
    _check(load().rp_entry_grad(h.ptr, _ptr(lam), _ptr(x), _ptr(g_buffer), _stream(stream)), "rp_entry_grad")


def face_grad(h: Handle, lam, x, g_face, stream=None):
    _check(load().rp_face_grad(h.ptr, _ptr(lam), _ptr(x), _ptr(g_face), _stream(stream)), "rp_face_grad")


def check_violations(reset: bool = False):
    """rp_check_violations (bounds-checked library only): (accesses skipped,
    first site, first index) since the last reset; waits for the device."""
    c, site, idx = ctypes.c_uint64(), ctypes.c_int32(), ctypes.c_int64()
    _check(load().rp_check_violations(ctypes.byref(c), ctypes.byref(site), ctypes.byref(idx), int(reset)),
           "rp_check_violations")
    return c.value, site.value, idx.value


@dataclasses.dataclass
class Exports:
    """Names the header declares (checked against the loaded library)."""
    names: tuple = ("rp_default_options", "rp_build_repartition", "rp_get_part_map", "rp_get_sizes",
                    "rp_update_values_packed", "rp_update_values", "rp_get_values", "rp_spmv", "rp_solve",
                    "rp_solve_adjoint", "rp_profile_iteration", "rp_entry_grad", "rp_face_grad", "rp_destroy", "rp_status_str",
                    "rp_last_error", "rp_spmv_noalloc", "rp_batch_build", "rp_batch_update_solve",
                    "rp_batch_set_config", "rp_batch_autotune", "rp_set_solver_options", "rp_iter_spmv",
                    "rp_get_sliced_view", "rp_solve_bicgstab", "rp_solve_bicgstab_mixed", "rp_get_solve_info",
                    "rp_check_violations")
