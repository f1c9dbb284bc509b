"""The C ABI loads, exports what include/repart.h declares, and rejects
malformed descriptors on the host before any device work (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2510_08536_gb300 import build, repart, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return repart.load()


def _declared():
    txt = open(os.path.join(ROOT, "include", "repart.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(rp_[a-z_0-9]+)\s*\(", txt)))


def test_header_symbols_exported(lib):
    names = _declared()
    assert "rp_build_repartition" in names and "rp_solve" in names
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) <= set(repart.Exports().names)


def test_status_strings(lib):
    assert lib.rp_status_str(0) == b"RP_OK"
    assert lib.rp_status_str(repart.RP_EDUP) == b"RP_EDUP"
    assert lib.rp_status_str(repart.RP_BREAKDOWN) == b"RP_BREAKDOWN"


def test_default_options(lib):
    o = repart.default_options()
    assert o.n_parts == 1 and o.want_fp32 == 1 and o.max_iter > 0 and o.inner_tol == 1e-5


class _R:
    def __init__(self, **kw):
        self.__dict__.update(kw)


def _ranks():
    m = synth.box_mesh(4, 3, 2, 2, 1, 1)
    return [_R(n_cells=r.n_cells, lower_addr=r.lower_addr.copy(), upper_addr=r.upper_addr.copy(),
               iface_row=r.iface_row.copy(), iface_nbr_rank=r.iface_nbr_rank.copy(),
               iface_nbr_col=r.iface_nbr_col.copy()) for r in m.ranks]


def _status(ranks, **kw):
    with pytest.raises(repart.RepartError) as e:
        repart.build_repartition(ranks, **kw)
    return e.value.status


def test_rejects_bad_descriptors(lib):
    r = _ranks()
    r[0].lower_addr[0] = r[0].upper_addr[0]
    assert _status(r) == repart.RP_EINVAL          # owner must be below neighbour
    r = _ranks()
    r[1].upper_addr[0] = r[1].n_cells
    assert _status(r) == repart.RP_ERANGE          # address outside the rank
    r = _ranks()
    r[0].iface_nbr_rank[0] = 0
    assert _status(r) == repart.RP_EINVAL          # interface to itself
    r = _ranks()
    r[0].iface_nbr_rank[0] = 5
    assert _status(r) == repart.RP_ERANGE          # unknown neighbour rank
    r = _ranks()
    r[0].iface_nbr_col[0] = (r[0].iface_nbr_col[0] + 1) % r[1].n_cells
    assert _status(r) == repart.RP_EINVAL          # interfaces not paired
    r = _ranks()
    r[1].iface_nbr_col[0] = r[0].n_cells + 3
    assert _status(r) == repart.RP_ERANGE
    assert _status(_ranks(), n_parts=3) == repart.RP_EINVAL  # n_parts must divide k
    r = _ranks()
    r[0].n_cells = -1
    assert _status(r) == repart.RP_EINVAL


def test_rejects_index_overflow(lib):
    big = _R(n_cells=2**31 - 100, lower_addr=np.zeros(0, np.int32), upper_addr=np.zeros(0, np.int32),
             iface_row=np.zeros(0, np.int32), iface_nbr_rank=np.zeros(0, np.int32),
             iface_nbr_col=np.zeros(0, np.int32))
    assert _status([big]) == repart.RP_EOVERFLOW


def test_null_arguments(lib):
    assert lib.rp_build_repartition(None, 0, None, None) == repart.RP_EINVAL
    assert lib.rp_solve(None, None, None, 1e-9, 0, 0, 0, None, None) == repart.RP_EINVAL
    assert lib.rp_update_values_packed(None, None, 0, None) == repart.RP_EINVAL
    assert b"null" in lib.rp_last_error()
    lib.rp_destroy(None)  # no-op


def test_batch_rejects_coupled_systems(lib):
    """Batched systems are independent: a system with interface entries is refused on the host."""
    with pytest.raises(repart.RepartError) as e:
        lib_ranks = _ranks()
        descs = (repart.LduDesc * len(lib_ranks))()
        keep = []
        for i, r in enumerate(lib_ranks):
            arrs = [np.ascontiguousarray(getattr(r, f), dtype=np.int32) for f in
                    ("lower_addr", "upper_addr", "iface_row", "iface_nbr_rank", "iface_nbr_col")]
            keep.append(arrs)
            p = [a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)) for a in arrs]
            descs[i] = repart.LduDesc(r.n_cells, arrs[0].size, p[0], p[1], arrs[2].size, p[2], p[3], p[4])
        out = ctypes.c_void_p()
        repart._check(lib.rp_batch_build(descs, len(lib_ranks), None, ctypes.byref(out)), "rp_batch_build")
    assert e.value.status == repart.RP_EINVAL
    assert b"interface" in lib.rp_last_error()
    assert lib.rp_batch_set_config(None, 8, 256) == repart.RP_EINVAL


def test_rejects_bad_solver_choices(lib):
    assert _status(_ranks(), layout=2) == repart.RP_EINVAL
    assert _status(_ranks(), precond=2) == repart.RP_EINVAL
    assert _status(_ranks(), spare=1) == repart.RP_EINVAL
    assert _status(_ranks(), n_parts=2, precond=repart.RP_PRECOND_LINE) == repart.RP_EUNSUPPORTED
    o = repart.default_options()
    assert o.precond == repart.RP_PRECOND_JACOBI and o.layout == repart.RP_LAYOUT_AUTO and o.spare == 0


def test_null_handle_solvers(lib):
    """Every solver entry point rejects a null handle on the host (RP_EINVAL)."""
    info = repart.SolveInfo()
    for name in ("rp_solve_bicgstab", "rp_solve_bicgstab_mixed"):
        st = getattr(lib, name)(None, None, None, 1e-9, 0, 0, ctypes.byref(info), None)
        assert st == repart.RP_EINVAL, name


def test_binding_rejects_unknown_precision(lib):
    import torch
    b = torch.zeros(4, dtype=torch.float64)
    with pytest.raises(ValueError):
        repart.solve_bicgstab(None, b, b.clone(), precision="fp16")


def test_get_solve_info_rejects_null(lib):
    info = repart.SolveInfo()
    assert lib.rp_get_solve_info(None, ctypes.byref(info), None) == repart.RP_EINVAL
    assert lib.rp_get_solve_info(None, None, None) == repart.RP_EINVAL


def test_update_rejects_unknown_where(lib):
    assert lib.rp_update_values_packed(None, None, repart.RP_MEM_HOST_ASYNC, None) == repart.RP_EINVAL


def test_check_violations_needs_the_checked_build(lib):
    """The normal library answers RP_EUNSUPPORTED with a zero count; the
    bounds-checked variant (built next to it) exports the same symbols."""
    c, site, idx = ctypes.c_uint64(7), ctypes.c_int32(7), ctypes.c_int64(7)
    st = lib.rp_check_violations(ctypes.byref(c), ctypes.byref(site), ctypes.byref(idx), 0)
    assert st == repart.RP_EUNSUPPORTED and c.value == 0 and site.value == 0 and idx.value == -1
    assert lib.rp_check_violations(None, None, None, 0) == repart.RP_EINVAL
    path = build.build(check=True)
    chk = ctypes.CDLL(path)
    for name in _declared():
        assert hasattr(chk, name), name
