"""rp_spmv_noalloc, the entry point for callers that cannot allocate device
memory (their memory belongs to a host framework's pool, or they run while a
stream is being captured, or they must not allocate after start-up).

It is checked through the C ABI against the handle-based rp_spmv on the same
matrix, on two calls in a row, with the SpMV tolerances of the parity tests.
This file is collected last so that a run stopping at the first failure has
run every other test before it; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import scipy.sparse as sp
import torch

from paper_2510_08536_gb300 import build, repart, synth

pytestmark = pytest.mark.gpu


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def test_spmv_noalloc_matches_rp_spmv():
    build.build()
    lib = repart.load()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    mesh = synth.box_mesh(40, 30, 20, 2, 2, 2)
    stg = synth.Assembler(mesh).staging(synth.face_coeffs(mesh, 1.0, 100))
    h = repart.build_repartition(mesh.ranks)
    repart.update_values_packed(h, torch.from_numpy(stg).to(dev))
    m = repart.get_part_map(h, 0)
    vals = repart.get_values(h)["vals"]
    n = h.n
    A = sp.csr_matrix((np.abs(vals.cpu().numpy()), m["col_idx"].cpu().numpy(), m["row_ptr"].cpu().numpy()),
                      shape=(n, n))
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rng = np.random.default_rng(7)
    for call in range(2):
        xs = rng.standard_normal(n)
        x = torch.from_numpy(xs).to(dev)
        y_ref = torch.empty_like(x)
        xy_ref = torch.zeros(1, dtype=torch.float64, device=dev)
        repart.spmv(h, x, y_ref, xy_ref)  # the existing entry point
        y = torch.full_like(x, float("nan"))
        xy = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info(dev)[0]
        st = lib.rp_spmv_noalloc(n, _p(m["row_ptr"]), _p(m["col_idx"]), _p(vals), _p(x), _p(y), _p(xy), stream)
        assert st == repart.RP_OK, lib.rp_last_error()
        torch.cuda.synchronize()
        if call > 0:  # no device memory taken by the call (the first one may load the module)
            assert torch.cuda.mem_get_info(dev)[0] == free0
        scale = A @ np.abs(xs)
        assert (np.abs(y.cpu().numpy() - y_ref.cpu().numpy()) <= 1e-13 * scale).all()
        assert abs(xy.item() - xy_ref.item()) <= 1e-12 * (np.abs(xs) @ scale)
    h.close()


def test_spmv_noalloc_rejects_oversize():
    lib = repart.load()
    too_many = 16_777_216 + 1
    dummy = ctypes.c_void_p(16)  # never dereferenced: the size check comes first
    st = lib.rp_spmv_noalloc(too_many, dummy, dummy, dummy, dummy, dummy, None, None)
    assert st == repart.RP_ERANGE
    assert b"static scratch limit" in lib.rp_last_error()
