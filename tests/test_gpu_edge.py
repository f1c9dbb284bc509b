"""Degenerate inputs on the GPU path against the oracle.

* A CPU rank with no cells between two others (the merged matrix is
  block-diagonal): maps bit-exact, one part and one part per rank (an empty
  part), the sliced layout built around it, FP64 and mixed solves as the
  oracle's.
* A system with no cells at all: every call succeeds and does nothing.
* A single cell without faces (a 1 x 1 matrix): one iteration, x = b / a.
"""
import types

import numpy as np
import pytest
import torch

from oracle import repart_oracle as O
from paper_2510_08536_gb300 import build, repart, synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    repart.load()
    torch.cuda.set_device(0)


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _empty_rank():
    z = np.zeros(0, np.int32)
    return types.SimpleNamespace(n_cells=0, n_faces=0, n_iface=0, lower_addr=z, upper_addr=z, iface_row=z,
                                 iface_nbr_rank=z, iface_nbr_col=z)


def _three_ranks():
    m1, m2 = synth.box_mesh(6, 5, 4, 1, 1, 1), synth.box_mesh(5, 4, 3, 1, 1, 1)
    s1 = synth.Assembler(m1).staging(synth.face_coeffs(m1, 0.5, 100))
    s2 = synth.Assembler(m2).staging(synth.face_coeffs(m2, 0.5, 101))
    ranks = [m1.ranks[0], _empty_rank(), m2.ranks[0]]
    return ranks, np.concatenate([s1, s2])


@pytest.mark.parametrize("n_parts", [1, 3])
def test_empty_rank_between_others(n_parts):
    ranks, stg = _three_ranks()
    n = sum(int(r.n_cells) for r in ranks)
    h = repart.build_repartition(ranks, n_parts=n_parts)
    parts = O.repartition_map(ranks, n_parts)
    for p, m in enumerate(parts):
        got = repart.get_part_map(h, p)
        assert got["n_rows"] == m.row_ptr.shape[0] - 1
        for key in ("row_ptr", "col_idx", "src_of", "diag_pos"):
            np.testing.assert_array_equal(got[key].cpu().numpy(), getattr(m, key), err_msg=f"{p} {key}")
    view = repart.get_sliced_view(h)
    assert view is not None
    assert view["n_slices"] == sum((m.row_ptr.shape[0] - 1 + 31) // 32 for m in parts)
    repart.update_values_packed(h, _t(stg))
    (m1,) = O.repartition_map(ranks, 1)
    vals = O.update_values(m1.src_of, stg)
    A = O.csr_matrix(m1.row_ptr, m1.col_idx, vals)
    b = np.random.default_rng(0).uniform(-1.0, 1.0, n)
    ref = O.pcg(A, O.jacobi_inverse(m1.row_ptr, m1.col_idx, vals, m1.diag_pos), b, tol=1e-9)
    for precision in ("fp64", "mixed", "mixed_ru"):
        x = torch.zeros(n, dtype=torch.float64, device=DEV)
        info = repart.solve(h, _t(b), x, tol=1e-9, precision=precision)
        xs = x.cpu().numpy()
        assert info["status"] == 0, (precision, info)
        assert np.linalg.norm(b - A @ xs) / np.linalg.norm(b) <= 1e-9
        if precision == "fp64":
            assert np.linalg.norm(xs - ref.x) / np.linalg.norm(ref.x) <= 1e-7
            assert abs(info["iterations"] - ref.iterations) <= 2
    h.close()


def test_system_without_cells():
    h = repart.build_repartition([_empty_rank()])
    assert h.n == 0 and repart.get_sliced_view(h) is None
    e = torch.zeros(0, dtype=torch.float64, device=DEV)
    repart.update_values_packed(h, e)
    for precision in ("fp64", "mixed", "mixed_ru"):
        info = repart.solve(h, e, torch.zeros(0, dtype=torch.float64, device=DEV), precision=precision)
        assert info["status"] == 0 and info["iterations"] == 0
    info = repart.solve_bicgstab(h, e, torch.zeros(0, dtype=torch.float64, device=DEV))
    assert info["status"] == 0 and info["iterations"] == 0
    h.close()


def test_single_cell():
    z = np.zeros(0, np.int32)
    rank = types.SimpleNamespace(n_cells=1, n_faces=0, n_iface=0, lower_addr=z, upper_addr=z, iface_row=z,
                                 iface_nbr_rank=z, iface_nbr_col=z)
    h = repart.build_repartition([rank])
    repart.update_values_packed(h, _t(np.array([4.0])))
    for precision in ("fp64", "mixed", "mixed_ru"):
        x = torch.zeros(1, dtype=torch.float64, device=DEV)
        info = repart.solve(h, _t(np.array([2.0])), x, tol=1e-9, precision=precision)
        assert info["status"] == 0 and abs(float(x[0]) - 0.5) <= 1e-15, (precision, info, float(x[0]))
    h.close()
