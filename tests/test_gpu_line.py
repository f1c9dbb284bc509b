"""PCG with the line (block-tridiagonal, 32-row blocks) preconditioner against the oracle.

* FP64: after exactly k = 1, 2, 5 iterations the GPU iterate equals the oracle's
  (same recurrence, preconditioner applied by a banded LU solve there, by warp
  scans here) to 1e-11 relative -- a direct check of the applied M^-1; at
  convergence ||x - x_ref|| / ||x_ref|| <= 1e-7, true residual <= 1e-9,
  iterations within 2.
* Mixed (FP32 factors, FP64 refinement): true FP64 residual <= 1e-9; inner
  iterations <= 1.25 x the oracle's (FP32 banded solve) + 10.
* On a line-ordered mesh the line preconditioner needs fewer iterations than Jacobi.
* Switching the preconditioner of a handle reproduces a handle built with it
  (bitwise); the host-launched loop reproduces the graph (bitwise).
"""
import numpy as np
import pytest
import torch

from oracle import repart_oracle as O
from paper_2510_08536_gb300 import build, repart, synth

from gpu_util import Case

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
LINE = repart.RP_PRECOND_LINE


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    repart.load()
    torch.cuda.set_device(0)


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _line_op(c, dtype=np.float64):
    vals = c.vals if dtype == np.float64 else O.to_fp32(c.vals)
    return O.line_operator(*O.line_part(c.map.row_ptr, c.map.col_idx, vals), dtype=dtype)


MESHES = [
    ((32, 16, 8), (1, 1, 1)),    # one rank, x-lines of 32 rows
    ((64, 32, 16), (2, 2, 1)),   # 4 ranks of 32 x 16 x 16: lines of 32
    ((13, 7, 9), (3, 2, 1)),     # ragged ranks: blocks cut across lines
]


@pytest.mark.parametrize("dims,parts", MESHES)
def test_line_fp64_iterates_match_oracle(dims, parts):
    c = Case(dims, parts, sigma=1.0)
    op = _line_op(c)
    for k in (1, 2, 5):
        h = repart.build_repartition(c.mesh.ranks, precond=LINE, max_iter=k, max_restarts=0)
        repart.update_values_packed(h, _t(c.staging))
        x = torch.zeros(c.mesh.n_cells, dtype=torch.float64, device=DEV)
        info = repart.solve(h, _t(c.b), x, tol=1e-14)
        ref = O.pcg(c.A, op, c.b, tol=1e-14, max_iter=k)
        assert info["iterations"] == k == ref.iterations
        assert np.linalg.norm(x.cpu().numpy() - ref.x) / np.linalg.norm(ref.x) <= 1e-11, k
        h.close()


@pytest.mark.parametrize("dims,parts", MESHES)
def test_line_fp64_solve_parity(dims, parts):
    c = Case(dims, parts, sigma=1.0)
    h = repart.build_repartition(c.mesh.ranks, precond=LINE)
    repart.update_values_packed(h, _t(c.staging))
    x = torch.zeros(c.mesh.n_cells, dtype=torch.float64, device=DEV)
    info = repart.solve(h, _t(c.b), x, tol=1e-9)
    ref = O.pcg(c.A, _line_op(c), c.b, tol=1e-9)
    xs = x.cpu().numpy()
    assert info["status"] == 0 and c.true_rel_residual(xs) <= 1e-9
    assert np.linalg.norm(xs - ref.x) / np.linalg.norm(ref.x) <= 1e-7
    assert abs(info["iterations"] - ref.iterations) <= 2
    h.close()


@pytest.mark.parametrize("precision", ["mixed", "mixed_ru"])
def test_line_mixed_solves(precision):
    c = Case((64, 32, 16), (2, 2, 1), sigma=1.0)
    h = repart.build_repartition(c.mesh.ranks, precond=LINE)
    repart.update_values_packed(h, _t(c.staging))
    x = torch.zeros(c.mesh.n_cells, dtype=torch.float64, device=DEV)
    info = repart.solve(h, _t(c.b), x, tol=1e-9, precision=precision)
    assert info["status"] == 0 and c.true_rel_residual(x.cpu().numpy()) <= 1e-9
    A32 = O.csr_matrix(c.map.row_ptr, c.map.col_idx, O.to_fp32(c.vals))
    op32 = _line_op(c, np.float32)
    if precision == "mixed_ru":
        ref = O.mixed_reliable(c.A, A32, op32, c.b, tol=1e-9, delta=0.1)
    else:
        ref = O.mixed_ir(c.A, A32, op32, c.b, tol=1e-9, inner_tol=1e-5)
    assert ref.status == O.OK
    assert info["iterations"] <= 1.25 * ref.iterations + 10, (info, ref.iterations)
    h.close()


def test_line_needs_fewer_iterations_than_jacobi():
    c = Case((64, 32, 16), (2, 2, 1), sigma=1.0, oracle_map=False)
    its = {}
    for name, pc in (("jacobi", repart.RP_PRECOND_JACOBI), ("line", LINE)):
        h = repart.build_repartition(c.mesh.ranks, precond=pc)
        repart.update_values_packed(h, _t(c.staging))
        for precision in ("fp64", "mixed_ru"):
            x = torch.zeros(c.mesh.n_cells, dtype=torch.float64, device=DEV)
            info = repart.solve(h, _t(c.b), x, tol=1e-9, precision=precision)
            assert info["status"] == 0
            its[name, precision] = info["iterations"]
        h.close()
    for precision in ("fp64", "mixed_ru"):
        assert its["line", precision] < 0.95 * its["jacobi", precision], its


def test_line_switch_and_host_loop_are_bitwise():
    c = Case((32, 16, 8), (1, 1, 1), sigma=1.0, oracle_map=False)
    b = _t(c.b)

    def run(h, precision):
        x = torch.zeros(c.mesh.n_cells, dtype=torch.float64, device=DEV)
        info = repart.solve(h, b, x, tol=1e-9, precision=precision)
        return x, info

    built = repart.build_repartition(c.mesh.ranks, precond=LINE)
    switched = repart.build_repartition(c.mesh.ranks)
    loop = repart.build_repartition(c.mesh.ranks, precond=LINE, host_loop=1)
    for h in (built, switched, loop):
        repart.update_values_packed(h, _t(c.staging))
    jac = {p: run(switched, p) for p in ("fp64", "mixed_ru")}
    repart.set_solver_options(switched, precond=LINE)
    for precision in ("fp64", "mixed", "mixed_ru"):
        xb, ib = run(built, precision)
        xs, is_ = run(switched, precision)
        xl, il = run(loop, precision)
        assert ib == is_ == il and ib["status"] == 0
        assert torch.equal(xb, xs) and torch.equal(xb, xl)
    # and back to Jacobi
    repart.set_solver_options(switched, precond=repart.RP_PRECOND_JACOBI)
    for p, (xj, ij) in jac.items():
        x, info = run(switched, p)
        assert info == ij and torch.equal(x, xj)
    for h in (built, switched, loop):
        h.close()


def test_line_rejects_multiple_parts():
    c = Case((16, 8, 8), (2, 1, 1), oracle_map=False)
    with pytest.raises(repart.RepartError) as e:
        repart.build_repartition(c.mesh.ranks, n_parts=2, precond=LINE)
    assert e.value.status == repart.RP_EUNSUPPORTED
    h = repart.build_repartition(c.mesh.ranks, n_parts=2)
    with pytest.raises(repart.RepartError) as e:
        repart.set_solver_options(h, precond=LINE)
    assert e.value.status == repart.RP_EUNSUPPORTED
    h.close()
