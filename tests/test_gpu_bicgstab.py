"""rp_solve_bicgstab (Jacobi-preconditioned BiCGStab, FP64) and
rp_solve_bicgstab_mixed (FP32 inner BiCGStab in FP64 refinement) against the oracle.

Tolerances: the oracle runs the same recurrence to the same tolerance, so
||x - x_ref|| / ||x_ref|| <= 1e-7 at rel. residual 1e-9 (summation order and
FMA contraction differ); the true residual of the GPU result, recomputed with
the oracle's matrix, <= 1e-9; iteration counts within max(3, 10%) of the
oracle's. Sliced and CSR layouts give bitwise-identical solves (same
products, same grids at these sizes). Mixed: the true FP64 residual <= 1e-9,
the solution within 1e-7 of the FP64 one, inner iterations at most 1.25 x the
oracle's (FP32 rounding order differs) + 10.
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


class Mom:
    """A momentum system: mesh, staging, the oracle's matrix, Jacobi inverse and rhs."""

    def __init__(self, dims, parts, seed=100):
        self.mesh = synth.box_mesh(*dims, *parts)
        self.stg = synth.momentum_staging(self.mesh, 0.5, seed)
        (self.map,) = O.repartition_map(self.mesh.ranks, 1)
        vals = O.update_values(self.map.src_of, self.stg)
        self.vals = vals
        self.A = O.csr_matrix(self.map.row_ptr, self.map.col_idx, vals)
        self.dinv = O.jacobi_inverse(self.map.row_ptr, self.map.col_idx, vals, self.map.diag_pos)
        self.b = synth.uniform_vector(self.mesh, 0)
        self.n = self.mesh.n_cells

    def true_rel(self, x):
        return float(np.linalg.norm(self.b - self.A @ x) / np.linalg.norm(self.b))

    def mixed_ref(self, inner_tol=1e-5):
        v32 = O.to_fp32(self.vals)
        A32 = O.csr_matrix(self.map.row_ptr, self.map.col_idx, v32)
        return O.bicgstab_mixed_ir(self.A, A32, np.float32(1) / v32[self.map.diag_pos], self.b, tol=1e-9,
                                   inner_tol=inner_tol)


MESHES = [
    ((32, 32, 32), (2, 2, 2)),
    ((13, 7, 9), (3, 2, 1)),
    ((10, 9, 8), (1, 1, 1)),
    ((40, 3, 2), (4, 1, 1)),
]


def _solve(h, b, n, tol=1e-9, **kw):
    x = torch.zeros(n, dtype=torch.float64, device=DEV)
    info = repart.solve_bicgstab(h, b, x, tol=tol, **kw)
    return x, info


@pytest.mark.parametrize("dims,parts", MESHES)
def test_bicgstab_parity(dims, parts):
    M = Mom(dims, parts)
    h = repart.build_repartition(M.mesh.ranks)
    repart.update_values_packed(h, _t(M.stg))
    x, info = _solve(h, _t(M.b), M.n)
    ref = O.bicgstab(M.A, M.dinv, M.b, tol=1e-9)
    xs = x.cpu().numpy()
    assert info["status"] == 0 and ref.status == O.OK, info
    assert M.true_rel(xs) <= 1e-9
    assert abs(info["rel_residual"] - M.true_rel(xs)) <= 1e-12
    assert np.linalg.norm(xs - ref.x) / np.linalg.norm(ref.x) <= 1e-7
    assert abs(info["iterations"] - ref.iterations) <= max(3, ref.iterations // 10), (info, ref.iterations)
    h.close()


def test_bicgstab_layouts_agree_bitwise():
    M = Mom((24, 20, 16), (2, 2, 1))
    hs = repart.build_repartition(M.mesh.ranks)
    hc = repart.build_repartition(M.mesh.ranks, layout=repart.RP_LAYOUT_CSR)
    assert repart.get_sliced_view(hs) is not None and repart.get_sliced_view(hc) is None
    out = []
    for h in (hs, hc):
        repart.update_values_packed(h, _t(M.stg))
        out.append(_solve(h, _t(M.b), M.n))
    assert out[0][1] == out[1][1] and out[0][1]["status"] == 0
    assert torch.equal(out[0][0], out[1][0])
    hs.close()
    hc.close()


@pytest.mark.parametrize("n_parts", [2, 4])
def test_bicgstab_multi_part(n_parts):
    M = Mom((16, 12, 10), (2, 2, 1))
    h = repart.build_repartition(M.mesh.ranks, n_parts=n_parts)
    repart.update_values_packed(h, _t(M.stg))
    x, info = _solve(h, _t(M.b), M.n)
    ref = O.bicgstab(M.A, M.dinv, M.b, tol=1e-9)
    xs = x.cpu().numpy()
    assert info["status"] == 0 and M.true_rel(xs) <= 1e-9
    assert np.linalg.norm(xs - ref.x) / np.linalg.norm(ref.x) <= 1e-7
    h.close()


def test_bicgstab_edge_cases():
    M = Mom((12, 10, 8), (2, 1, 1))
    h = repart.build_repartition(M.mesh.ranks, max_iter=5000)
    repart.update_values_packed(h, _t(M.stg))
    # b = 0: x = 0, no iterations
    x = torch.full((M.n,), 3.0, dtype=torch.float64, device=DEV)
    info = repart.solve_bicgstab(h, torch.zeros(M.n, dtype=torch.float64, device=DEV), x)
    assert info["status"] == 0 and info["iterations"] == 0 and not x.any()
    # the exact solution as a guess: converged before any iteration
    x = _t(np.linalg.solve(M.A.toarray(), M.b))
    info = repart.solve_bicgstab(h, _t(M.b), x, tol=1e-9, x_is_guess=True)
    assert info["status"] == 0 and info["iterations"] == 0
    # a guess that is not the solution
    x0 = np.random.default_rng(9).uniform(-1, 1, M.n)
    x = _t(x0)
    info = repart.solve_bicgstab(h, _t(M.b), x, tol=1e-9, x_is_guess=True)
    ref = O.bicgstab(M.A, M.dinv, M.b, tol=1e-9, x0=x0)
    assert info["status"] == 0 and M.true_rel(x.cpu().numpy()) <= 1e-9
    assert abs(info["iterations"] - ref.iterations) <= max(3, ref.iterations // 10)
    # host buffers give the device result
    xh = torch.zeros(M.n, dtype=torch.float64)
    info_h = repart.solve_bicgstab(h, torch.from_numpy(M.b.copy()), xh, tol=1e-9)
    xd, info_d = _solve(h, _t(M.b), M.n)
    assert info_h == info_d and torch.equal(xh, xd.cpu())
    h.close()
    # iteration cap
    h = repart.build_repartition(M.mesh.ranks, max_iter=4, max_restarts=0)
    repart.update_values_packed(h, _t(M.stg))
    x, info = _solve(h, _t(M.b), M.n, tol=1e-12)
    ref = O.bicgstab(M.A, M.dinv, M.b, tol=1e-12, max_iter=4)
    assert info["status"] == repart.RP_NOT_CONVERGED and info["iterations"] == 4
    assert np.linalg.norm(x.cpu().numpy() - ref.x) / np.linalg.norm(ref.x) <= 1e-10
    h.close()


def test_bicgstab_diagonal_system_one_step():
    n = 300
    z = np.zeros(0, np.int32)
    rank = types.SimpleNamespace(n_cells=n, lower_addr=z, upper_addr=z, iface_row=z, iface_nbr_rank=z,
                                 iface_nbr_col=z)
    d = np.random.default_rng(3).uniform(1.0, 5.0, n)
    b = np.random.default_rng(4).uniform(-1.0, 1.0, n)
    h = repart.build_repartition([rank])
    repart.update_values_packed(h, _t(d))
    x, info = _solve(h, _t(b), n)
    assert info["status"] == 0 and info["iterations"] == 1
    np.testing.assert_allclose(x.cpu().numpy(), b / d, rtol=1e-15)
    h.close()


def test_bicgstab_on_spd_matches_pcg_solution():
    """On the SPD pressure matrix BiCGStab and CG reach the same solution."""
    mesh = synth.box_mesh(16, 16, 16, 2, 2, 2)
    stg = synth.Assembler(mesh).staging(synth.face_coeffs(mesh, 0.5, 100))
    b = _t(synth.uniform_vector(mesh, 0))
    h = repart.build_repartition(mesh.ranks)
    repart.update_values_packed(h, _t(stg))
    xb, ib = _solve(h, b, mesh.n_cells, tol=1e-11)
    xc = torch.zeros_like(xb)
    ic = repart.solve(h, b, xc, tol=1e-11)
    assert ib["status"] == 0 and ic["status"] == 0
    assert float(torch.linalg.norm(xb - xc) / torch.linalg.norm(xc)) <= 1e-8
    h.close()


@pytest.mark.parametrize("dims,parts", MESHES)
def test_bicgstab_mixed_parity(dims, parts):
    M = Mom(dims, parts)
    h = repart.build_repartition(M.mesh.ranks)
    repart.update_values_packed(h, _t(M.stg))
    x, info = _solve(h, _t(M.b), M.n, precision="mixed")
    ref = M.mixed_ref()
    xs = x.cpu().numpy()
    assert info["status"] == 0 and ref.status == O.OK, info
    assert M.true_rel(xs) <= 1e-9
    assert abs(info["rel_residual"] - M.true_rel(xs)) <= 1e-12
    ref64 = O.bicgstab(M.A, M.dinv, M.b, tol=1e-12)
    assert np.linalg.norm(xs - ref64.x) / np.linalg.norm(ref64.x) <= 1e-7
    assert info["outer_iterations"] >= 1
    assert info["iterations"] <= 1.25 * ref.iterations + 10, (info, ref.iterations, ref.outer_iterations)
    h.close()


def test_bicgstab_mixed_layouts_parts_and_edges():
    M = Mom((24, 20, 16), (2, 2, 1))
    hs = repart.build_repartition(M.mesh.ranks)
    hc = repart.build_repartition(M.mesh.ranks, layout=repart.RP_LAYOUT_CSR)
    hp = repart.build_repartition(M.mesh.ranks, n_parts=2)
    out = []
    for h in (hs, hc, hp):
        repart.update_values_packed(h, _t(M.stg))
        out.append(_solve(h, _t(M.b), M.n, precision="mixed"))
    assert out[0][1] == out[1][1] and out[0][1]["status"] == 0
    assert torch.equal(out[0][0], out[1][0])  # the same products and reductions on both layouts
    assert out[2][1]["status"] == 0 and M.true_rel(out[2][0].cpu().numpy()) <= 1e-9
    # b = 0: x = 0 without iterations; host buffers give the device result
    x = torch.full((M.n,), 2.0, dtype=torch.float64, device=DEV)
    info = repart.solve_bicgstab(hs, torch.zeros(M.n, dtype=torch.float64, device=DEV), x, precision="mixed")
    assert info["status"] == 0 and info["iterations"] == 0 and not x.any()
    xh = torch.zeros(M.n, dtype=torch.float64)
    info_h = repart.solve_bicgstab(hs, torch.from_numpy(M.b.copy()), xh, tol=1e-9, precision="mixed")
    assert info_h == out[0][1] and torch.equal(xh, out[0][0].cpu())
    for h in (hs, hc, hp):
        h.close()
    h = repart.build_repartition(M.mesh.ranks, want_fp32=False)
    with pytest.raises(repart.RepartError) as e:
        repart.solve_bicgstab(h, _t(M.b), torch.zeros(M.n, dtype=torch.float64, device=DEV), precision="mixed")
    assert e.value.status == repart.RP_EINVAL
    h.close()



def test_bicgstab_host_loop_matches_graph():
    """The host-launched loop (for profilers) runs the graph's kernels in the same
    order: the same bits in both precisions."""
    M = Mom((20, 16, 12), (2, 2, 1))
    out = {}
    for host_loop in (0, 1):
        h = repart.build_repartition(M.mesh.ranks, host_loop=host_loop)
        repart.update_values_packed(h, _t(M.stg))
        for precision in ("fp64", "mixed"):
            out[host_loop, precision] = _solve(h, _t(M.b), M.n, precision=precision)
        h.close()
    for precision in ("fp64", "mixed"):
        (xg, ig), (xl, il) = out[0, precision], out[1, precision]
        assert ig == il and ig["status"] == 0, precision
        assert torch.equal(xg, xl), precision
