"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Maps and value updates are compared bit for bit; floating-point results
within the tolerances stated next to each assertion:
  * SpMV: |y - y_ref| <= 1e-13 * (|A| |x|)_i per row (rounding of <= 7 terms
    in a different order, FMA contraction);
  * FP64 PCG to rel. residual 1e-9: the true residual of the GPU result
    <= 1e-9 and ||x - x_ref|| / ||x_ref|| <= 1e-7 against the oracle PCG run
    with the same tolerance (same recurrence, different summation order);
  * mixed: true FP64 residual <= 1e-9; error vs the FP64 oracle <= 1e-6.
"""
import numpy as np
import pytest
import torch

from oracle import repart_oracle as O
from paper_2510_08536_gb300 import build, repart, synth

from gpu_util import Case

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    repart.load()
    torch.cuda.set_device(0)


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


MESHES = [
    ((32, 32, 32), (2, 2, 2)),   # the 32^3, k=8 plain FP64 workload
    ((13, 7, 9), (3, 2, 1)),     # uneven split, ragged tails
    ((10, 9, 8), (1, 1, 1)),     # k = 1
    ((40, 3, 2), (4, 1, 1)),     # thin slab ranks
    ((2, 1, 1), (2, 1, 1)),      # two cells, one interface (alpha = 2)
]


# ------------------------------------------------------------------ map


@pytest.mark.parametrize("dims,parts", MESHES)
@pytest.mark.parametrize("symmetric", [False, True])
def test_map_bit_exact(dims, parts, symmetric):
    mesh = synth.box_mesh(*dims, *parts)
    h = repart.build_repartition(mesh.ranks, symmetric=symmetric, want_transpose=True)
    (m,) = O.repartition_map(mesh.ranks, 1, symmetric)
    got = repart.get_part_map(h, 0)
    for key in ("row_ptr", "col_idx", "src_of", "diag_pos", "tpos"):
        np.testing.assert_array_equal(got[key].cpu().numpy(), getattr(m, key), err_msg=key)
    assert got["nl_nnz"] == 0 and got["n_nl_cols"] == 0
    h.close()


@pytest.mark.parametrize("n_parts", [2, 4, 8])
def test_map_multi_part_bit_exact(n_parts):
    mesh = synth.box_mesh(16, 12, 8, 2, 2, 2)
    h = repart.build_repartition(mesh.ranks, n_parts=n_parts, want_transpose=True)
    parts = O.repartition_map(mesh.ranks, n_parts)
    for p, m in enumerate(parts):
        got = repart.get_part_map(h, p)
        assert got["row_off"] == m.row_off and got["buf_off"] == m.buf_off and got["buf_len"] == m.buf_len
        for key in ("row_ptr", "col_idx", "src_of", "diag_pos", "tpos", "nl_row_ptr", "nl_col_idx",
                    "nl_src_of", "nl_cols"):
            np.testing.assert_array_equal(got[key].cpu().numpy(), getattr(m, key), err_msg=f"part {p} {key}")
    h.close()


@pytest.mark.parametrize("n_parts", [2, 4, 8])
def test_multi_part_spmv_and_solve(n_parts):
    """Solving over the parts' local + non-local matrices (halo gathered on the
    device) gives the merged system's product and solution."""
    c = Case((24, 20, 16), (2, 2, 2), sigma=1.0)
    h1 = repart.build_repartition(c.mesh.ranks)
    hp = repart.build_repartition(c.mesh.ranks, n_parts=n_parts)
    assert hp.n_parts == n_parts
    stg = _t(c.staging)
    repart.update_values_packed(h1, stg)
    repart.update_values_packed(hp, stg)
    n = c.mesh.n_cells
    x = np.random.default_rng(4).standard_normal(n)
    y = torch.empty(n, dtype=torch.float64, device=DEV)
    repart.spmv(hp, _t(x), y)
    ref = O.spmv(c.map.row_ptr, c.map.col_idx, c.vals, x)
    scale = O.spmv(c.map.row_ptr, c.map.col_idx, np.abs(c.vals), np.abs(x))
    assert (np.abs(y.cpu().numpy() - ref) <= 1e-13 * scale).all()
    for precision in ("fp64", "mixed", "mixed_ru"):
        x1 = torch.zeros(n, dtype=torch.float64, device=DEV)
        xp = torch.zeros_like(x1)
        i1 = repart.solve(h1, _t(c.b), x1, tol=1e-9, precision=precision)
        ip = repart.solve(hp, _t(c.b), xp, tol=1e-9, precision=precision)
        assert ip["status"] == 0, ip
        xs = xp.cpu().numpy()
        assert c.true_rel_residual(xs) <= 1e-9
        assert np.linalg.norm(xs - x1.cpu().numpy()) / np.linalg.norm(xs) <= 1e-6
        if precision == "fp64":
            assert abs(ip["iterations"] - i1["iterations"]) <= 2
    h1.close()
    hp.close()


def test_duplicate_face_rejected_on_device():
    mesh = synth.box_mesh(4, 3, 3, 2, 1, 1)
    r = mesh.ranks[1]
    r.lower_addr = np.concatenate([r.lower_addr, r.lower_addr[2:3]])
    r.upper_addr = np.concatenate([r.upper_addr, r.upper_addr[2:3]])
    with pytest.raises(repart.RepartError) as e:
        repart.build_repartition(mesh.ranks)
    assert e.value.status == repart.RP_EDUP


# ------------------------------------------------------------------ values


@pytest.mark.parametrize("symmetric", [False, True])
def test_update_bit_exact(symmetric):
    c = Case((24, 20, 16), (3, 2, 2), sigma=1.0, symmetric=symmetric)
    h = repart.build_repartition(c.mesh.ranks, symmetric=symmetric)
    repart.update_values_packed(h, _t(c.staging))
    v = repart.get_values(h)
    np.testing.assert_array_equal(v["vals"].cpu().numpy(), c.vals)
    np.testing.assert_array_equal(v["vals32"].cpu().numpy(), O.to_fp32(c.vals))
    np.testing.assert_array_equal(v["dinv"].cpu().numpy(), c.dinv)
    # a second draw through host memory and through per-rank arrays
    stg2 = c.asm.staging(synth.face_coeffs(c.mesh, 1.0, 101))
    repart.update_values_packed(h, torch.from_numpy(stg2).pin_memory())
    np.testing.assert_array_equal(repart.get_values(h)["vals"].cpu().numpy(), O.update_values(c.map.src_of, stg2))
    sl = c.asm.rank_slices(c.staging)
    for dev in (True, False):
        conv = (lambda a: _t(a)) if dev else (lambda a: torch.from_numpy(np.ascontiguousarray(a)))
        repart.update_values(h, [conv(s[0]) for s in sl], [conv(s[1]) for s in sl],
                             None if symmetric else [conv(s[2]) for s in sl], [conv(s[3]) for s in sl])
        np.testing.assert_array_equal(repart.get_values(h)["vals"].cpu().numpy(), c.vals)
    h.close()


def test_update_reads_host_memory_in_place():
    """RP_MEM_HOST_DIRECT: the permutation kernel gathers from host memory over
    the CPU-GPU link; the values are the same bits as from a device buffer."""
    c = Case((24, 20, 16), (3, 2, 2), sigma=1.0)
    h = repart.build_repartition(c.mesh.ranks)
    repart.update_values_packed(h, torch.from_numpy(c.staging).pin_memory(), direct=True)
    v = repart.get_values(h)
    np.testing.assert_array_equal(v["vals"].cpu().numpy(), c.vals)
    np.testing.assert_array_equal(v["dinv"].cpu().numpy(), c.dinv)
    # pageable memory: read in place where the device can (Grace), refused otherwise
    stg2 = c.asm.staging(synth.face_coeffs(c.mesh, 1.0, 101))
    try:
        repart.update_values_packed(h, torch.from_numpy(stg2), direct=True)
    except repart.RepartError as e:
        assert e.status == repart.RP_EUNSUPPORTED
    else:
        np.testing.assert_array_equal(repart.get_values(h)["vals"].cpu().numpy(),
                                      O.update_values(c.map.src_of, stg2))
    h.close()


def test_spmv_parity():
    c = Case((30, 20, 17), (3, 2, 1), sigma=1.0)
    h = repart.build_repartition(c.mesh.ranks)
    repart.update_values_packed(h, _t(c.staging))
    x = np.random.default_rng(3).standard_normal(c.mesh.n_cells)
    y = torch.empty(c.mesh.n_cells, dtype=torch.float64, device=DEV)
    xy = torch.zeros(1, dtype=torch.float64, device=DEV)
    repart.spmv(h, _t(x), y, xy)
    ref = O.spmv(c.map.row_ptr, c.map.col_idx, c.vals, x)
    scale = O.spmv(c.map.row_ptr, c.map.col_idx, np.abs(c.vals), np.abs(x))
    assert (np.abs(y.cpu().numpy() - ref) <= 1e-13 * scale).all()
    assert abs(xy.item() - x @ ref) <= 1e-12 * (np.abs(x) @ scale)
    h.close()


# ------------------------------------------------------------------ solves


@pytest.mark.parametrize("dims,parts,sigma", [
    ((32, 32, 32), (2, 2, 2), None),     # the plain FP64 workload
    ((24, 24, 24), (2, 3, 1), 0.5),
    ((33, 17, 9), (3, 1, 3), 1.0),
])
def test_fp64_solve_parity(dims, parts, sigma):
    c = Case(dims, parts, sigma=sigma)
    h = repart.build_repartition(c.mesh.ranks)
    repart.update_values_packed(h, _t(c.staging))
    ref = O.pcg(c.A, c.dinv, c.b, tol=1e-9)
    x = torch.zeros(c.mesh.n_cells, dtype=torch.float64, device=DEV)
    info = repart.solve(h, _t(c.b), x, tol=1e-9)
    xs = x.cpu().numpy()
    assert info["status"] == repart.RP_OK, info
    assert c.true_rel_residual(xs) <= 1e-9
    assert abs(info["rel_residual"] - c.true_rel_residual(xs)) <= 1e-3 * 1e-9
    assert np.linalg.norm(xs - ref.x) / np.linalg.norm(ref.x) <= 1e-7
    assert abs(info["iterations"] - ref.iterations) <= 2, (info, ref.iterations)
    # a second solve gives the same bits (deterministic reductions)
    x2 = torch.zeros_like(x)
    repart.solve(h, _t(c.b), x2, tol=1e-9)
    assert torch.equal(x, x2)
    h.close()


def _inner_count_ok(got, oracle, fp64):
    """Inner FP32 iteration counts depend on rounding order (the kernels sum dot
    products per thread in FP32, the oracle in FP64), by several percent either
    way: no fewer than exact PCG needs (95% of the FP64 count, less 5) and no
    more than 10% above the oracle's form (+ 10). A lost correction or a wrong
    recurrence costs far more."""
    assert 0.95 * fp64 - 5 <= got <= 1.10 * oracle + 10, (got, oracle, fp64)


def _scaled_system(c):
    """The oracle's scaling s = fl32(1/sqrt(a_ii)) and FP32 matrix S A S."""
    s_ = O.jacobi_scaling(c.vals[c.map.diag_pos])
    return s_, O.csr_matrix(c.map.row_ptr, c.map.col_idx,
                            O.scaled_fp32_values(c.map.row_ptr, c.map.col_idx, c.vals, s_))


def test_mixed_solve_parity():
    c = Case((32, 32, 32), (2, 2, 2), sigma=1.0)
    h = repart.build_repartition(c.mesh.ranks)
    repart.update_values_packed(h, _t(c.staging))
    x = torch.zeros(c.mesh.n_cells, dtype=torch.float64, device=DEV)
    info = repart.solve(h, _t(c.b), x, tol=1e-9, precision="mixed")
    xs = x.cpu().numpy()
    assert info["status"] == repart.RP_OK, info
    assert info["outer_iterations"] >= 2
    assert c.true_rel_residual(xs) <= 1e-9
    # the inner FP32 iteration runs on S A S (sliced layout, one part, Jacobi)
    s_, Ah32 = _scaled_system(c)
    ref = O.mixed_ir_scaled(c.A, Ah32, s_, c.b, tol=1e-9)
    assert ref.status == O.OK
    x64 = O.pcg(c.A, c.dinv, c.b, tol=1e-12).x
    assert np.linalg.norm(xs - x64) / np.linalg.norm(x64) <= 1e-6
    assert abs(info["outer_iterations"] - ref.outer_iterations) <= 1
    # the inner FP32 recurrence: total inner iterations as the oracle's, and the
    # last pass stops near the target like the oracle's (half of it), not far below
    _inner_count_ok(info["iterations"], ref.iterations, O.pcg(c.A, c.dinv, c.b, tol=1e-9).iterations)
    assert 1e-10 <= info["rel_residual"] <= 1e-9 and 1e-10 <= ref.true_rel_residual <= 1e-9
    h.close()


@pytest.mark.parametrize("sigma", [None, 1.0])
def test_mixed_continued_solve_parity(sigma):
    """RP_MIXED_RU against the oracle's refinement with a continued inner PCG."""
    c = Case((32, 32, 32), (2, 2, 2), sigma=sigma)
    h = repart.build_repartition(c.mesh.ranks)
    repart.update_values_packed(h, _t(c.staging))
    x = torch.zeros(c.mesh.n_cells, dtype=torch.float64, device=DEV)
    info = repart.solve(h, _t(c.b), x, tol=1e-9, precision="mixed_ru")
    xs = x.cpu().numpy()
    assert info["status"] == repart.RP_OK, info
    assert c.true_rel_residual(xs) <= 1e-9
    s_, Ah32 = _scaled_system(c)
    ref = O.mixed_reliable_scaled(c.A, Ah32, s_, c.b, tol=1e-9, delta=0.1)
    assert ref.status == O.OK
    x64 = O.pcg(c.A, c.dinv, c.b, tol=1e-12).x
    assert np.linalg.norm(xs - x64) / np.linalg.norm(x64) <= 1e-6
    _inner_count_ok(info["iterations"], ref.iterations, O.pcg(c.A, c.dinv, c.b, tol=1e-9).iterations)
    h.close()


def test_solve_edge_cases():
    c = Case((12, 10, 8), (2, 2, 1), sigma=0.5)
    h = repart.build_repartition(c.mesh.ranks, max_iter=5000)
    repart.update_values_packed(h, _t(c.staging))
    n = c.mesh.n_cells
    # b = 0 -> x = 0, no iterations
    x = torch.full((n,), 7.0, dtype=torch.float64, device=DEV)
    info = repart.solve(h, torch.zeros(n, dtype=torch.float64, device=DEV), x)
    assert info["status"] == 0 and info["iterations"] == 0 and not x.any()
    # the exact solution as a guess -> converged before any iteration
    xe = np.linalg.solve(c.A.toarray(), c.b)
    x = _t(xe)
    info = repart.solve(h, _t(c.b), x, tol=1e-9, x_is_guess=True)
    assert info["status"] == 0 and info["iterations"] == 0
    h.close()
    # iteration cap
    h = repart.build_repartition(c.mesh.ranks, max_iter=3, max_restarts=0)
    repart.update_values_packed(h, _t(c.staging))
    x = torch.zeros(n, dtype=torch.float64, device=DEV)
    info = repart.solve(h, _t(c.b), x, tol=1e-12)
    assert info["status"] == repart.RP_NOT_CONVERGED and info["iterations"] == 3
    ref = O.pcg(c.A, c.dinv, c.b, tol=1e-12, max_iter=3)
    assert np.linalg.norm(x.cpu().numpy() - ref.x) / np.linalg.norm(ref.x) <= 1e-12
    h.close()
    # a negative definite matrix breaks down (p.Ap <= 0) instead of looping
    h = repart.build_repartition(c.mesh.ranks)
    repart.update_values_packed(h, _t(-c.staging))
    x = torch.zeros(n, dtype=torch.float64, device=DEV)
    info = repart.solve(h, _t(c.b), x, tol=1e-9)
    assert info["status"] == repart.RP_BREAKDOWN
    info = repart.solve(h, _t(c.b), x, tol=1e-9, precision="mixed")
    assert info["status"] == repart.RP_BREAKDOWN
    h.close()


def test_host_buffers_match_device():
    c = Case((20, 16, 12), (2, 2, 1), sigma=1.0)
    h = repart.build_repartition(c.mesh.ranks)
    repart.update_values_packed(h, torch.from_numpy(c.staging).pin_memory())
    xd = torch.zeros(c.mesh.n_cells, dtype=torch.float64, device=DEV)
    repart.solve(h, _t(c.b), xd)
    xh = torch.zeros(c.mesh.n_cells, dtype=torch.float64).pin_memory()
    info = repart.solve(h, torch.from_numpy(c.b).pin_memory(), xh)
    assert info["status"] == 0
    assert torch.equal(xd.cpu(), xh)
    h.close()


# ------------------------------------------------------------------ adjoint


@pytest.mark.parametrize("symmetric", [False, True])
def test_adjoint_and_gradients(symmetric):
    c = Case((16, 12, 10), (2, 2, 2), sigma=0.5, symmetric=symmetric)
    h = repart.build_repartition(c.mesh.ranks, symmetric=symmetric, want_transpose=True)
    repart.update_values_packed(h, _t(c.staging))
    n = c.mesh.n_cells
    x = torch.zeros(n, dtype=torch.float64, device=DEV)
    repart.solve(h, _t(c.b), x, tol=1e-12)
    xt = synth.uniform_vector(c.mesh, 1)
    g = x - _t(xt)
    lam = torch.zeros_like(x)
    info = repart.solve_adjoint(h, g, lam, tol=1e-12)
    assert info["status"] == 0
    AT = O.csr_matrix(c.map.row_ptr, c.map.col_idx, O.transpose_values(c.vals, c.map.tpos))
    lam_ref = np.linalg.solve(AT.toarray(), g.cpu().numpy())
    lam_np = lam.cpu().numpy()
    assert np.linalg.norm(lam_np - lam_ref) / np.linalg.norm(lam_ref) <= 1e-9
    gb = torch.zeros(h.n_slots, dtype=torch.float64, device=DEV)
    repart.entry_grad(h, lam, x, gb)
    ge = O.entry_grad(c.map.row_ptr, c.map.col_idx, lam_np, x.cpu().numpy())
    ref = O.slot_grad(c.map.src_of, ge, h.n_slots)
    np.testing.assert_allclose(gb.cpu().numpy(), ref, rtol=1e-14, atol=0)
    nf = sum(r.n_faces + r.n_iface for r in c.mesh.ranks)
    gf = torch.zeros(nf, dtype=torch.float64, device=DEV)
    repart.face_grad(h, lam, x, gf)
    np.testing.assert_allclose(gf.cpu().numpy(), O.face_grad_ldu(c.mesh.ranks, lam_np, x.cpu().numpy()),
                               rtol=1e-14, atol=0)
    h.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed_ru"])
def test_host_loop_matches_graph(precision):
    """The profiler-friendly host-driven loop runs the graph's kernels in the same order."""
    c = Case((20, 18, 16), (2, 2, 2), sigma=1.0, oracle_map=False)
    outs = []
    for host_loop in (0, 1):
        h = repart.build_repartition(c.mesh.ranks, host_loop=host_loop)
        repart.update_values_packed(h, _t(c.staging))
        x = torch.zeros(c.mesh.n_cells, dtype=torch.float64, device=DEV)
        info = repart.solve(h, _t(c.b), x, tol=1e-9, precision=precision)
        assert info["status"] == 0
        outs.append((x.cpu(), info))
        h.close()
    assert torch.equal(outs[0][0], outs[1][0])
    assert outs[0][1] == outs[1][1]
