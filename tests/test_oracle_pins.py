"""Pins of the CPU oracle against facts that do not come from the oracle.

Each test ties one oracle function to something independent: a
hand-enumerated map, a different library construction, a dense solve, a
closed form, an invariant written another way, or finite differences.
"""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import repart_oracle as O
from paper_2510_08536_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


# ---------------------------------------------------------------- maps


@pytest.mark.parametrize("case", ["two_cells_k2", "four_cells_k2"])
def test_hand_enumerated_alpha2(case):
    g = _golden("alpha2_maps.json")[case]
    mesh = synth.box_mesh(*g["mesh"], *g["ranks"])
    (m,) = O.repartition_map(mesh.ranks, 1)
    e = g["n_parts_1"]
    for key in ("row_ptr", "col_idx", "src_of", "diag_pos", "tpos"):
        np.testing.assert_array_equal(getattr(m, key), e[key], err_msg=key)
    assert m.nl_col_idx.size == 0
    if "n_parts_2" in g:
        parts = O.repartition_map(mesh.ranks, 2)
        for m, e in zip(parts, g["n_parts_2"]):
            for key, v in e.items():
                np.testing.assert_array_equal(getattr(m, key), v, err_msg=key)


def _scipy_csr(mesh, symmetric):
    """Independent construction: scipy COO -> CSR of (row, col, slot+1)."""
    off = np.cumsum([0] + [r.n_cells for r in mesh.ranks])
    rows, cols, slots = [], [], []
    s = 0
    for ri, r in enumerate(mesh.ranks):
        n, f, e = r.n_cells, r.n_faces, r.n_iface
        rows += list(off[ri] + np.arange(n)); cols += list(off[ri] + np.arange(n)); slots += list(s + np.arange(n))
        rows += list(off[ri] + r.lower_addr); cols += list(off[ri] + r.upper_addr); slots += list(s + n + np.arange(f))
        lslot = s + n + np.arange(f) if symmetric else s + n + f + np.arange(f)
        rows += list(off[ri] + r.upper_addr); cols += list(off[ri] + r.lower_addr); slots += list(lslot)
        base = s + n + (1 if symmetric else 2) * f
        rows += list(off[ri] + r.iface_row); cols += list(off[r.iface_nbr_rank] + r.iface_nbr_col)
        slots += list(base + np.arange(e))
        s = base + e
    n = off[-1]
    m = sp.coo_matrix((np.array(slots, np.float64) + 1, (rows, cols)), shape=(n, n)).tocsr()
    m.sort_indices()
    return m


@pytest.mark.parametrize("dims,parts,symmetric", [
    ((6, 5, 4), (2, 1, 2), False),
    ((7, 3, 5), (3, 1, 1), True),
    ((5, 6, 7), (1, 3, 2), False),
    ((9, 4, 3), (2, 2, 1), True),
])
def test_map_equals_scipy_coo_to_csr(dims, parts, symmetric):
    mesh = synth.box_mesh(*dims, *parts)
    (m,) = O.repartition_map(mesh.ranks, 1, symmetric)
    ref = _scipy_csr(mesh, symmetric)
    np.testing.assert_array_equal(m.row_ptr, ref.indptr)
    np.testing.assert_array_equal(m.col_idx, ref.indices)
    np.testing.assert_array_equal(m.src_of, ref.data.astype(np.int64) - 1)
    # the transposed position really holds the transposed entry
    n = m.n_rows
    row_of = np.repeat(np.arange(n), np.diff(m.row_ptr))
    assert (m.tpos >= 0).all()
    np.testing.assert_array_equal(row_of[m.tpos], m.col_idx)
    np.testing.assert_array_equal(m.col_idx[m.tpos], row_of)
    np.testing.assert_array_equal(m.col_idx[m.diag_pos], np.arange(n))


def test_nonlocal_split_partitions_every_entry():
    """With n_parts > 1 every entry lands in exactly one of the local or
    non-local matrices of its owning part, with the right global column."""
    mesh = synth.box_mesh(8, 6, 4, 4, 2, 1)
    ref = _scipy_csr(mesh, False).tocoo()
    want = set(zip(ref.row.tolist(), ref.col.tolist(), (ref.data.astype(int) - 1).tolist()))
    got = set()
    for pm in O.repartition_map(mesh.ranks, 4):
        row_of = np.repeat(np.arange(pm.n_rows), np.diff(pm.row_ptr))
        got |= set(zip((row_of + pm.row_off).tolist(), (pm.col_idx + pm.row_off).tolist(),
                       (pm.src_of + pm.buf_off).tolist()))
        nrow = np.repeat(np.arange(pm.n_rows), np.diff(pm.nl_row_ptr))
        gcol = pm.nl_cols[pm.nl_col_idx]
        assert ((gcol < pm.row_off) | (gcol >= pm.row_off + pm.n_rows)).all()
        assert (np.diff(pm.nl_cols) > 0).all()
        got |= set(zip((nrow + pm.row_off).tolist(), gcol.tolist(), (pm.nl_src_of + pm.buf_off).tolist()))
    assert got == want


def test_fewer_parts_fewer_nonlocal_entries():
    """Sec. 3: repartitioning into fewer parts leaves fewer non-local coefficients."""
    mesh = synth.box_mesh(8, 8, 8, 2, 2, 2)
    counts = [sum(pm.nl_col_idx.size for pm in O.repartition_map(mesh.ranks, p)) for p in (8, 4, 2, 1)]
    assert counts[0] > counts[1] > counts[2] > counts[3] == 0


def test_row_entries_match_full_map():
    mesh = synth.box_mesh(7, 6, 5, 2, 3, 1)
    for symmetric in (False, True):
        (m,) = O.repartition_map(mesh.ranks, 1, symmetric)
        for row in [0, 1, 17, 41, mesh.n_cells - 1]:
            s, e = m.row_ptr[row], m.row_ptr[row + 1]
            want = list(zip(m.col_idx[s:e].tolist(), m.src_of[s:e].tolist()))
            assert O.row_entries(mesh.ranks, row, symmetric) == want


def test_duplicate_entry_rejected():
    mesh = synth.box_mesh(3, 2, 2)
    r = mesh.ranks[0]
    r.lower_addr = np.concatenate([r.lower_addr, r.lower_addr[:1]])
    r.upper_addr = np.concatenate([r.upper_addr, r.upper_addr[:1]])
    with pytest.raises(ValueError):
        O.repartition_map(mesh.ranks, 1)


# ---------------------------------------------------------------- values


def _dense_physical(mesh, a, shift=synth.DIAG_SHIFT):
    """The physical matrix in GLOBAL cell order, straight from the faces."""
    nx, ny, nz = mesh.nx, mesh.ny, mesh.nz
    n = mesh.n_cells
    A = np.zeros((n, n))
    gid = lambda i, j, k: i + nx * (j + ny * k)
    f = 0
    for k in range(nz):
        for j in range(ny):
            for i in range(nx - 1):
                c1, c2 = gid(i, j, k), gid(i + 1, j, k)
                A[c1, c2] -= a[f]; A[c2, c1] -= a[f]; A[c1, c1] += a[f]; A[c2, c2] += a[f]; f += 1
    for k in range(nz):
        for j in range(ny - 1):
            for i in range(nx):
                c1, c2 = gid(i, j, k), gid(i, j + 1, k)
                A[c1, c2] -= a[f]; A[c2, c1] -= a[f]; A[c1, c1] += a[f]; A[c2, c2] += a[f]; f += 1
    for k in range(nz - 1):
        for j in range(ny):
            for i in range(nx):
                c1, c2 = gid(i, j, k), gid(i, j, k + 1)
                A[c1, c2] -= a[f]; A[c2, c1] -= a[f]; A[c1, c1] += a[f]; A[c2, c2] += a[f]; f += 1
    for k in range(nz):
        for j in range(ny):
            c = gid(0, j, k)
            A[c, c] += 2 * a[f]; f += 1
    A += shift * np.eye(n)
    return A


@pytest.mark.parametrize("symmetric", [False, True])
def test_updated_values_form_the_physical_matrix(symmetric):
    mesh = synth.box_mesh(5, 4, 3, 2, 2, 1)
    a = synth.face_coeffs(mesh, 0.5, 7)
    stg = synth.Assembler(mesh, symmetric).staging(a)
    (m,) = O.repartition_map(mesh.ranks, 1, symmetric)
    vals = O.update_values(m.src_of, stg)
    merged = O.csr_matrix(m.row_ptr, m.col_idx, vals).toarray()
    gid = mesh.merged_gid()
    A = _dense_physical(mesh, a)
    np.testing.assert_allclose(merged, A[np.ix_(gid, gid)], rtol=1e-14, atol=1e-14)
    v32 = O.to_fp32(vals)
    assert v32.dtype == np.float32 and np.array_equal(v32, vals.astype(np.float32))


@pytest.mark.parametrize("symmetric", [False, True])
def test_spmv_equals_sum_of_ldu_products(symmetric):
    mesh = synth.box_mesh(9, 7, 6, 3, 1, 2)
    a = synth.face_coeffs(mesh, 1.0, 3)
    stg = synth.Assembler(mesh, symmetric).staging(a)
    (m,) = O.repartition_map(mesh.ranks, 1, symmetric)
    x = np.random.default_rng(5).standard_normal(mesh.n_cells)
    y_csr = O.spmv(m.row_ptr, m.col_idx, O.update_values(m.src_of, stg), x)
    y_ldu = O.ldu_matvec(mesh.ranks, stg, x, symmetric)
    np.testing.assert_allclose(y_csr, y_ldu, rtol=1e-13, atol=1e-13)


# ---------------------------------------------------------------- solves


def _system(mesh, sigma, seed=100, symmetric=False):
    a = synth.face_coeffs(mesh, sigma, seed)
    stg = synth.Assembler(mesh, symmetric).staging(a)
    (m,) = O.repartition_map(mesh.ranks, 1, symmetric)
    vals = O.update_values(m.src_of, stg)
    A = O.csr_matrix(m.row_ptr, m.col_idx, vals)
    dinv = O.jacobi_inverse(m.row_ptr, m.col_idx, vals, m.diag_pos)
    return m, vals, A, dinv, a, stg


def test_pcg_matches_dense_solve():
    mesh = synth.box_mesh(10, 10, 10, 2, 2, 1)
    m, vals, A, dinv, _, _ = _system(mesh, 1.0)
    b = synth.uniform_vector(mesh, 0)
    res = O.pcg(A, dinv, b, tol=1e-12)
    assert res.status == O.OK and res.true_rel_residual <= 1e-12
    x = np.linalg.solve(A.toarray(), b)
    assert np.linalg.norm(res.x - x) / np.linalg.norm(x) < 1e-9


def _eig(mesh, m_, p_, q_):
    nx, ny, nz = mesh.nx, mesh.ny, mesh.nz
    lam = (4 * np.sin((2 * m_ + 1) * np.pi / (4 * nx)) ** 2 + 4 * np.sin(p_ * np.pi / (2 * ny)) ** 2
           + 4 * np.sin(q_ * np.pi / (2 * nz)) ** 2 + synth.DIAG_SHIFT)
    i = np.arange(nx) + 0.5
    j = np.arange(ny) + 0.5
    k = np.arange(nz) + 0.5
    v = (np.sin((2 * m_ + 1) * np.pi * i / (2 * nx))[None, None, :]
         * np.cos(p_ * np.pi * j / ny)[None, :, None] * np.cos(q_ * np.pi * k / nz)[:, None, None])
    return lam, v.ravel()


@pytest.mark.parametrize("mpq", [(0, 0, 0), (2, 1, 3), (5, 4, 0)])
def test_closed_form_eigenpairs(mpq):
    """Uniform 7-point operator, Dirichlet at x=0 (ghost cell), Neumann
    elsewhere: A v = lambda v, and PCG on b = v returns v / lambda."""
    mesh = synth.box_mesh(12, 10, 8, 2, 2, 2)
    m, vals, A, dinv, _, _ = _system(mesh, None)
    lam, vg = _eig(mesh, *mpq)
    v = vg[mesh.merged_gid()]
    np.testing.assert_allclose(A @ v, lam * v, rtol=0, atol=1e-13)
    res = O.pcg(A, dinv, v, tol=1e-13)
    assert res.status == O.OK
    np.testing.assert_allclose(res.x, v / lam, rtol=0, atol=1e-9 * np.abs(v / lam).max())


def test_manufactured_solution():
    mesh = synth.box_mesh(16, 12, 10, 2, 3, 2)
    m, vals, A, dinv, a, stg = _system(mesh, 0.5, seed=11)
    gid = mesh.merged_gid()
    gi, gj, gk = gid % mesh.nx, (gid // mesh.nx) % mesh.ny, gid // (mesh.nx * mesh.ny)
    xs = np.sin(0.3 * gi) * np.cos(0.2 * gj) + 0.1 * np.random.default_rng(2).standard_normal(gid.size) + gk * 0.01
    b = O.ldu_matvec(mesh.ranks, stg, xs)  # not through the CSR path
    res = O.pcg(A, dinv, b, tol=1e-13)
    assert res.status == O.OK
    assert np.linalg.norm(res.x - xs) / np.linalg.norm(xs) < 1e-9


def test_decomposition_invariance():
    sols = []
    for p in [(1, 1, 1), (2, 2, 2), (4, 4, 4)]:
        mesh = synth.box_mesh(16, 16, 16, *p)
        m, vals, A, dinv, _, _ = _system(mesh, 0.5)
        b = synth.uniform_vector(mesh, 0)
        res = O.pcg(A, dinv, b, tol=1e-12)
        xg = np.empty_like(res.x)
        xg[mesh.merged_gid()] = res.x
        sols.append((xg, res.iterations))
    for xg, it in sols[1:]:
        assert np.linalg.norm(xg - sols[0][0]) / np.linalg.norm(sols[0][0]) < 1e-10
        # same physical matrix, permuted: the CG recurrence is the same up to rounding
        assert abs(it - sols[0][1]) <= 2


def test_pcg_edge_cases():
    mesh = synth.box_mesh(4, 4, 4, 2, 1, 1)
    m, vals, A, dinv, _, _ = _system(mesh, 0.5)
    z = O.pcg(A, dinv, np.zeros(mesh.n_cells))
    assert z.status == O.OK and z.iterations == 0 and not z.x.any()
    b = synth.uniform_vector(mesh, 0)
    exact = np.linalg.solve(A.toarray(), b)
    warm = O.pcg(A, dinv, b, tol=1e-9, x0=exact)
    assert warm.status == O.OK and warm.iterations == 0
    lim = O.pcg(A, dinv, b, tol=1e-14, max_iter=3)
    assert lim.status == O.NOT_CONVERGED and lim.iterations == 3
    # an indefinite matrix breaks down (p.Ap <= 0)
    neg = O.pcg(-A, -dinv, b, tol=1e-9)
    assert neg.status == O.BREAKDOWN


def test_jacobi_inverse_is_reciprocal_diagonal():
    mesh = synth.box_mesh(5, 5, 5, 1, 1, 1)
    m, vals, A, dinv, _, _ = _system(mesh, 1.0)
    np.testing.assert_array_equal(dinv, 1.0 / A.diagonal())
    np.testing.assert_array_equal(O.jacobi_inverse(m.row_ptr, m.col_idx, vals), dinv)


def test_mixed_refinement_reaches_fp64_residual():
    mesh = synth.box_mesh(16, 16, 16, 2, 2, 2)
    m, vals, A, dinv, _, _ = _system(mesh, 1.0)
    v32 = O.to_fp32(vals)
    A32 = O.csr_matrix(m.row_ptr, m.col_idx, v32)
    dinv32 = np.float32(1.0) / v32[m.diag_pos]
    b = synth.uniform_vector(mesh, 0)
    res = O.mixed_ir(A, A32, dinv32, b, tol=1e-9, inner_tol=1e-5)
    assert res.status == O.OK and res.outer_iterations >= 2
    tr = np.linalg.norm(b - A @ res.x) / np.linalg.norm(b)
    assert tr <= 1e-9
    x = np.linalg.solve(A.toarray(), b)
    assert np.linalg.norm(res.x - x) / np.linalg.norm(x) < 1e-6
    # FP32 values alone cannot reach 1e-9: the FP64 outer residual is what gets there
    d, _, _ = O.pcg_fp32(A32, dinv32, b.astype(np.float32), 1e-7, 5000)
    assert np.linalg.norm(b - A @ d.astype(np.float64)) / np.linalg.norm(b) > 1e-9


def _system32(mesh, sigma):
    m, vals, A, dinv, _, _ = _system(mesh, sigma)
    v32 = O.to_fp32(vals)
    A32 = O.csr_matrix(m.row_ptr, m.col_idx, v32)
    return m, vals, A, dinv, A32, np.float32(1.0) / v32[m.diag_pos]


def test_pcg_fp32_in_fp64_is_the_fp64_recurrence():
    """The inner PCG of the restarted refinement run in FP64 from d = 0 is pcg
    itself: the same iterate after k iterations (a wrong beta, sign or step
    order would differ)."""
    mesh = synth.box_mesh(12, 10, 8, 2, 1, 1)
    m, vals, A, dinv, _, _ = _system(mesh, 1.0)
    b = synth.uniform_vector(mesh, 0)
    for k in (1, 2, 7, 20):
        d, it, st = O.pcg_fp32(A, dinv, b.copy(), rel_tol=0.0, max_iter=k, dtype=np.float64)
        ref = O.pcg(A, dinv, b, tol=0.0, max_iter=k)
        assert it == k == ref.iterations and st == O.NOT_CONVERGED
        assert np.linalg.norm(d - ref.x) / np.linalg.norm(ref.x) <= 1e-12, k


def test_pcg_fp32_iterates_match_scipy_cg_in_fp32():
    """In FP32 the inner PCG follows scipy's preconditioned CG run on the same
    FP32 matrix, right-hand side and Jacobi diagonal, iterate for iterate, up to
    FP32 rounding (scipy accumulates its dot products in FP32, the oracle in
    FP64; the recurrences are the same)."""
    import scipy.sparse.linalg as sla
    mesh = synth.box_mesh(12, 10, 8, 2, 1, 1)
    m, vals, A, dinv, A32, d32 = _system32(mesh, 1.0)
    b32 = synth.uniform_vector(mesh, 0).astype(np.float32)
    its = []
    M = sla.LinearOperator(A32.shape, matvec=lambda r: d32 * r, dtype=np.float32)
    sla.cg(A32, b32, rtol=1e-30, atol=0.0, maxiter=8, M=M, callback=lambda xk: its.append(xk.copy()))
    assert len(its) == 8 and its[0].dtype == np.float32
    for k in range(1, 9):
        d, it, st = O.pcg_fp32(A32, d32, b32.copy(), rel_tol=0.0, max_iter=k)
        assert d.dtype == np.float32 and it == k
        assert np.linalg.norm(d - its[k - 1]) / np.linalg.norm(its[k - 1]) <= 1e-5, k


def test_restarted_refinement_with_exact_inner_is_one_pcg_run():
    """With an FP64 inner solve the first refinement already solves the system:
    one outer pass, whose iterate is pcg's at the inner stopping point -- half
    the outer target (the last-pass bound), or inner_tol when the bound is off."""
    mesh = synth.box_mesh(12, 10, 8, 2, 1, 1)
    m, vals, A, dinv, _, _ = _system(mesh, 1.0)
    b = synth.uniform_vector(mesh, 0)
    for last_pass, ref_tol in ((0.5, 0.5e-9), (0.0, 1e-11)):
        one = O.mixed_ir(A, A, dinv, b, tol=1e-9, inner_tol=1e-11, dtype=np.float64, last_pass=last_pass)
        ref = O.pcg(A, dinv, b, tol=ref_tol)
        assert one.status == O.OK and one.outer_iterations == 1
        assert one.iterations == ref.iterations
        assert np.linalg.norm(one.x - ref.x) / np.linalg.norm(ref.x) <= 1e-12


def test_restarted_refinement_last_pass_stops_near_target():
    """The FP32 refinement's last pass stops at half the outer target instead of
    a further inner_tol reduction: the final FP64 residual sits within a decade
    below tol, with fewer inner iterations than the uncapped schedule."""
    mesh = synth.box_mesh(16, 16, 16, 2, 2, 2)
    m, vals, A, dinv, A32, d32 = _system32(mesh, 1.0)
    b = synth.uniform_vector(mesh, 0)
    capped = O.mixed_ir(A, A32, d32, b, tol=1e-9, inner_tol=1e-5)
    free = O.mixed_ir(A, A32, d32, b, tol=1e-9, inner_tol=1e-5, last_pass=0.0)
    for r in (capped, free):
        assert r.status == O.OK
        assert np.linalg.norm(b - A @ r.x) / np.linalg.norm(b) == pytest.approx(r.true_rel_residual, rel=1e-12)
    assert 1e-10 <= capped.true_rel_residual <= 1e-9
    assert free.true_rel_residual < capped.true_rel_residual
    assert capped.iterations < free.iterations and capped.outer_iterations == free.outer_iterations


def test_reliable_refinement_with_exact_inner_is_plain_pcg():
    """With FP64 inner arithmetic every replaced residual equals the recursive
    one up to rounding, so continuing the search direction must reproduce the
    plain PCG run (iterations and solution); a restart or a wrong beta after a
    replacement would not."""
    mesh = synth.box_mesh(16, 14, 12, 2, 2, 1)
    m, vals, A, dinv, _, _ = _system(mesh, 1.0)
    b = synth.uniform_vector(mesh, 0)
    ref = O.pcg(A, dinv, b, tol=1e-10)
    for delta in (1e-1, 1e-3, 1e-5):
        res = O.mixed_reliable(A, A, dinv, b, tol=1e-10, delta=delta, dtype=np.float64)
        assert res.status == O.OK
        # each replacement perturbs the residual by rounding only: at most ~1 extra iteration per two
        assert abs(res.iterations - ref.iterations) <= 2 + res.outer_iterations // 2, \
            (delta, res.iterations, ref.iterations, res.outer_iterations)
        assert np.linalg.norm(res.x - ref.x) / np.linalg.norm(ref.x) < 1e-8
        assert res.outer_iterations >= 1
    # restarting the search direction at every refinement costs far more
    # (the same steps with p = z after each replacement, written out here)
    f = np.float64
    x = np.zeros_like(b)
    total = 0
    for _ in range(50):
        res_ = b - A @ x
        if np.linalg.norm(res_) <= 1e-10 * np.linalg.norm(b):
            break
        d, it, _st = O.pcg_fp32(A, dinv, res_.astype(f), 1e-1, 10000, dtype=f)
        x += d
        total += it
    assert total > ref.iterations + 20


def test_reliable_refinement_fp32_reaches_fp64_residual():
    mesh = synth.box_mesh(16, 16, 16, 2, 2, 2)
    m, vals, A, dinv, _, _ = _system(mesh, 1.0)
    v32 = O.to_fp32(vals)
    A32 = O.csr_matrix(m.row_ptr, m.col_idx, v32)
    dinv32 = np.float32(1.0) / v32[m.diag_pos]
    b = synth.uniform_vector(mesh, 0)
    x = np.linalg.solve(A.toarray(), b)
    for delta in (1e-1, 1e-5):
        res = O.mixed_reliable(A, A32, dinv32, b, tol=1e-9, delta=delta)
        assert res.status == O.OK
        assert np.linalg.norm(b - A @ res.x) / np.linalg.norm(b) <= 1e-9
        assert np.linalg.norm(res.x - x) / np.linalg.norm(x) < 1e-6


# ---------------------------------------------------------------- adjoint


def test_transpose_values_give_dense_transpose():
    mesh = synth.box_mesh(4, 3, 3, 2, 1, 1)
    (m,) = O.repartition_map(mesh.ranks, 1)
    rng = np.random.default_rng(3)
    vals = rng.standard_normal(m.src_of.size)  # a general (non-symmetric) matrix
    A = O.csr_matrix(m.row_ptr, m.col_idx, vals).toarray()
    AT = O.csr_matrix(m.row_ptr, m.col_idx, O.transpose_values(vals, m.tpos)).toarray()
    np.testing.assert_array_equal(AT, A.T)


def test_gradients_by_central_differences():
    """L = 0.5 ||x - x_t||^2 with A x = b: dL/db = lambda and the face
    gradient -(lam_l - lam_u)(x_l - x_u) agree with central differences."""
    mesh = synth.box_mesh(6, 5, 4, 2, 1, 2)
    a = synth.face_coeffs(mesh, 0.5, 100)
    asm = synth.Assembler(mesh)
    b = synth.uniform_vector(mesh, 0)
    xt = synth.uniform_vector(mesh, 1)
    (m,) = O.repartition_map(mesh.ranks, 1)

    def solve(a_, b_):
        vals = O.update_values(m.src_of, asm.staging(a_))
        A = O.csr_matrix(m.row_ptr, m.col_idx, vals).toarray()
        return A, np.linalg.solve(A, b_)

    def loss(a_, b_):
        return 0.5 * float(np.sum((solve(a_, b_)[1] - xt) ** 2))

    A, x = solve(a, b)
    vals = O.update_values(m.src_of, asm.staging(a))
    AT = O.csr_matrix(m.row_ptr, m.col_idx, O.transpose_values(vals, m.tpos))
    lam = np.linalg.solve(AT.toarray(), x - xt)
    np.testing.assert_allclose(lam, np.linalg.solve(A, x - xt), rtol=1e-12, atol=1e-12)  # symmetric A
    h = 1e-6
    for i in [0, 7, 33, mesh.n_cells - 1]:
        e = np.zeros_like(b); e[i] = h
        fd = (loss(a, b + e) - loss(a, b - e)) / (2 * h)
        assert abs(fd - lam[i]) <= 1e-6 * max(1.0, abs(lam[i]))
    # face gradient through global face ids, interface faces included
    fg = O.face_grad_ldu(mesh.ranks, lam, x)
    fid = np.concatenate([np.concatenate([r.face_gid, r.iface_face_gid]) for r in mesh.ranks])
    for t in [0, 5, len(fid) // 2, len(fid) - 1]:
        f = fid[t]
        e = np.zeros_like(a); e[f] = h
        fd = (loss(a + e, b) - loss(a - e, b)) / (2 * h)
        assert abs(fd - fg[t]) <= 1e-6 * max(1.0, abs(fg[t]))
    # the entry gradient, summed per slot, reproduces the face gradient by the chain rule
    ge = O.entry_grad(m.row_ptr, m.col_idx, lam, x)
    gs = O.slot_grad(m.src_of, ge, asm.index.size)
    r0 = mesh.ranks[0]
    n0, f0 = r0.n_cells, r0.n_faces
    for f in range(f0):
        l, u = r0.lower_addr[f], r0.upper_addr[f]
        chain = gs[l] + gs[u] - gs[n0 + f] - gs[n0 + f0 + f]
        assert abs(chain - fg[f]) <= 1e-12 * max(1.0, abs(fg[f]))


# ---------------------------------------------------------------- BiCGStab (momentum)


def _momentum(dims, parts, seed=100):
    mesh = synth.box_mesh(*dims, *parts)
    stg = synth.momentum_staging(mesh, 0.5, seed)
    (m,) = O.repartition_map(mesh.ranks, 1)
    vals = O.update_values(m.src_of, stg)
    A = O.csr_matrix(m.row_ptr, m.col_idx, vals)
    dinv = O.jacobi_inverse(m.row_ptr, m.col_idx, vals, m.diag_pos)
    return mesh, stg, m, A, dinv, synth.uniform_vector(mesh, 0)


def test_momentum_matrix_rows_and_ldu_product():
    """The synthetic momentum matrix is non-symmetric with row sums ct, and the merged
    CSR product equals the per-rank LDU products with distinct lower / upper values."""
    mesh, stg, m, A, dinv, b = _momentum((9, 7, 6), (3, 1, 2))
    n = mesh.n_cells
    np.testing.assert_allclose(A @ np.ones(n), synth.MOMENTUM_CT, rtol=0, atol=1e-12)
    assert abs(A - A.T).max() > 0.1
    x = np.random.default_rng(5).standard_normal(n)
    np.testing.assert_allclose(A @ x, O.ldu_matvec(mesh.ranks, stg, x, False), rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("dims,parts", [((7, 6, 5), (2, 2, 1)), ((16, 16, 16), (2, 2, 2)), ((11, 9, 4), (1, 3, 1))])
def test_bicgstab_matches_scipy(dims, parts):
    """scipy.sparse.linalg.bicgstab with M = D^-1 is an independent implementation of
    the same recurrence: same iterate, same count (scipy does not count a final half step)."""
    import scipy.sparse.linalg as spl
    mesh, stg, m, A, dinv, b = _momentum(dims, parts)
    res = O.bicgstab(A, dinv, b, tol=1e-10)
    calls = []
    xs, info = spl.bicgstab(A, b, rtol=1e-10, atol=0.0, M=sp.diags(dinv), callback=lambda xk: calls.append(1))
    assert info == 0 and res.status == O.OK
    np.testing.assert_allclose(res.x, xs, rtol=1e-12, atol=1e-14)
    assert res.iterations - len(calls) in (0, 1)


def test_bicgstab_matches_dense_solve():
    mesh, stg, m, A, dinv, b = _momentum((6, 5, 4), (2, 1, 1))
    res = O.bicgstab(A, dinv, b, tol=1e-12)
    xe = np.linalg.solve(A.toarray(), b)
    assert res.status == O.OK and res.true_rel_residual <= 1e-12
    assert np.linalg.norm(res.x - xe) / np.linalg.norm(xe) <= 1e-10


def test_bicgstab_diagonal_system_is_one_step():
    """A = D: the Jacobi-preconditioned direction is the solution, alpha = 1 up to rounding."""
    d = np.random.default_rng(3).uniform(1.0, 5.0, 40)
    A = sp.csr_matrix(sp.diags(d))
    b = np.random.default_rng(4).uniform(-1.0, 1.0, 40)
    res = O.bicgstab(A, 1.0 / d, b, tol=1e-9)
    assert res.status == O.OK and res.iterations == 1
    np.testing.assert_allclose(res.x, b / d, rtol=1e-15)


def test_bicgstab_recursive_residual_tracks_true_residual():
    """x and r are updated consistently: after k iterations the recursive residual
    equals b - A x to rounding (a wrong sign or coefficient in either update breaks it)."""
    mesh, stg, m, A, dinv, b = _momentum((12, 10, 8), (2, 1, 1))
    for k in (1, 2, 5, 13, 30):
        res = O.bicgstab(A, dinv, b, tol=1e-14, max_iter=k)
        assert res.status == O.NOT_CONVERGED and res.iterations == k
        assert abs(res.rel_residual - res.true_rel_residual) <= 1e-12


def test_bicgstab_edge_cases():
    mesh, stg, m, A, dinv, b = _momentum((5, 4, 3), (1, 1, 1))
    res = O.bicgstab(A, dinv, np.zeros_like(b))
    assert res.status == O.OK and res.iterations == 0 and not res.x.any()
    xe = np.linalg.solve(A.toarray(), b)
    res = O.bicgstab(A, dinv, b, tol=1e-9, x0=xe)
    assert res.status == O.OK and res.iterations == 0


def test_bicgstab_fp32_inner_in_fp64_is_the_fp64_recurrence():
    """The inner solver run in FP64 from x0 = 0 is bicgstab itself: the same
    iterates after k iterations (a wrong step order, sign or scalar would differ)."""
    mesh, stg, m, A, dinv, b = _momentum((10, 8, 6), (2, 1, 1))
    for k in (1, 2, 7, 20):
        d, it, st = O.bicgstab_fp32(A, dinv, b.copy(), rel_tol=0.0, max_iter=k, dtype=np.float64)
        ref = O.bicgstab(A, dinv, b, tol=0.0, max_iter=k)
        assert it == k == ref.iterations and st == O.NOT_CONVERGED
        assert np.linalg.norm(d - ref.x) / np.linalg.norm(ref.x) <= 1e-12, k


def test_bicgstab_mixed_refinement_reaches_fp64_residual():
    """FP32 inner BiCGStab (FP32 values, vectors and products) inside FP64 refinement:
    the true FP64 residual reaches 1e-9 although one FP32 pass stalls near 1e-7, and the
    result agrees with the FP64 solve; with an FP64 inner solve one pass suffices."""
    mesh, stg, m, A, dinv, b = _momentum((14, 12, 10), (2, 2, 1))
    vals = O.update_values(m.src_of, stg)
    v32 = O.to_fp32(vals)
    A32 = O.csr_matrix(m.row_ptr, m.col_idx, v32)
    d32 = np.float32(1) / v32[m.diag_pos]
    res = O.bicgstab_mixed_ir(A, A32, d32, b, tol=1e-9, inner_tol=1e-5)
    assert res.status == O.OK and res.true_rel_residual <= 1e-9
    assert res.outer_iterations >= 2
    ref = O.bicgstab(A, dinv, b, tol=1e-12)
    assert np.linalg.norm(res.x - ref.x) / np.linalg.norm(ref.x) <= 1e-8
    one = O.bicgstab_mixed_ir(A, A, dinv, b, tol=1e-9, inner_tol=1e-11, dtype=np.float64)
    assert one.status == O.OK and one.outer_iterations == 1


def test_bicgstab_mixed_edge_cases():
    mesh, stg, m, A, dinv, b = _momentum((5, 4, 3), (1, 1, 1))
    A32 = A.astype(np.float32)
    res = O.bicgstab_mixed_ir(A, A32, dinv.astype(np.float32), np.zeros_like(b))
    assert res.status == O.OK and res.iterations == 0 and not res.x.any()
    d = np.random.default_rng(3).uniform(1.0, 5.0, 40)
    D = sp.csr_matrix(sp.diags(d))
    bd = np.random.default_rng(4).uniform(-1.0, 1.0, 40)
    res = O.bicgstab_mixed_ir(D, D.astype(np.float32), (1.0 / d).astype(np.float32), bd, tol=1e-9)
    # a diagonal system: every inner solve ends at its first half step
    assert res.status == O.OK and res.iterations == res.outer_iterations
    np.testing.assert_allclose(res.x, bd / d, rtol=1e-9)


# ---------------------------------------------------------------- line (block-tridiagonal) preconditioner


def _line_dense(A, block):
    """Independent construction: the dense matrix with every entry outside the
    diagonal and the in-block first off-diagonals set to zero."""
    D = A.toarray()
    n = D.shape[0]
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    keep = (i == j) | ((np.abs(i - j) == 1) & (i // block == j // block))
    return np.where(keep, D, 0.0)


@pytest.mark.parametrize("block", [32, 8])
def test_line_operator_is_block_tridiagonal_solve(block):
    mesh = synth.box_mesh(40, 3, 2, 2, 1, 1)
    m, vals, A, dinv, a, stg = _system(mesh, 1.0)
    sub, diag, sup = O.line_part(m.row_ptr, m.col_idx, vals, block)
    M = _line_dense(A, block)
    r = np.random.default_rng(2).standard_normal(mesh.n_cells)
    np.testing.assert_allclose(O.line_operator(sub, diag, sup)(r), np.linalg.solve(M, r), rtol=1e-11, atol=1e-13)
    assert np.linalg.eigvalsh(M).min() > 0.0  # SPD: a valid CG preconditioner


def test_line_pcg_is_exact_on_one_tridiagonal_block():
    mesh = synth.box_mesh(32, 1, 1, 1, 1, 1)
    m, vals, A, dinv, a, stg = _system(mesh, 1.0)
    b = synth.uniform_vector(mesh, 0)
    res = O.pcg(A, O.line_operator(*O.line_part(m.row_ptr, m.col_idx, vals)), b, tol=1e-12)
    assert res.status == O.OK and res.iterations == 1
    np.testing.assert_allclose(res.x, np.linalg.solve(A.toarray(), b), rtol=1e-10)


def test_line_pcg_beats_jacobi_on_line_ordered_box():
    mesh = synth.box_mesh(32, 16, 8, 1, 1, 1)   # rows x-fastest: x-lines of 32 rows
    m, vals, A, dinv, a, stg = _system(mesh, 1.0)
    b = synth.uniform_vector(mesh, 0)
    jac = O.pcg(A, dinv, b, tol=1e-9)
    line = O.pcg(A, O.line_operator(*O.line_part(m.row_ptr, m.col_idx, vals)), b, tol=1e-9)
    assert jac.status == O.OK and line.status == O.OK and line.true_rel_residual <= 1e-9
    assert line.iterations < 0.95 * jac.iterations
    xe = np.linalg.solve(A.toarray(), b)
    assert np.linalg.norm(line.x - xe) / np.linalg.norm(xe) <= 1e-6


def test_line_reliable_refinement_fp32_reaches_fp64_residual():
    mesh = synth.box_mesh(32, 12, 10, 1, 1, 1)
    m, vals, A, dinv, a, stg = _system(mesh, 1.0)
    b = synth.uniform_vector(mesh, 0)
    v32 = O.to_fp32(vals)
    A32 = O.csr_matrix(m.row_ptr, m.col_idx, v32)
    op32 = O.line_operator(*O.line_part(m.row_ptr, m.col_idx, v32), dtype=np.float32)
    res = O.mixed_reliable(A, A32, op32, b, tol=1e-9, delta=0.1)
    assert res.status == O.OK and res.true_rel_residual <= 1e-9


# ---------------------------------------------------------------- C / OpenMP restatement


@pytest.mark.parametrize("dims,parts,sigma", [((32, 32, 32), (2, 2, 2), None), ((24, 20, 18), (2, 2, 1), 1.0),
                                              ((7, 5, 3), (1, 1, 1), 0.5)])
def test_c_oracle_equals_python_oracle(dims, parts, sigma):
    """The C / OpenMP restatement (timed on all host cores by the benchmark) gives
    the Python oracle's update bit for bit and its PCG to rounding: the same
    iteration count and status, x within 1e-12, on one thread and on all."""
    from oracle import pcg_omp as C
    mesh = synth.box_mesh(*dims, *parts)
    m, vals, A, dinv, _, stg = _system(mesh, sigma)
    b = synth.uniform_vector(mesh, 0)
    ref = O.pcg(A, dinv, b, tol=1e-9)
    for th in (1, 0):
        v = C.update_values(m.src_of, stg, threads=th)
        np.testing.assert_array_equal(v, vals)
        d = C.jacobi_inverse(m.diag_pos, v, threads=th)
        np.testing.assert_array_equal(d, dinv)
        r = C.pcg(m.row_ptr, m.col_idx, v, d, b, tol=1e-9, threads=th)
        assert r.status == ref.status == O.OK and r.iterations == ref.iterations
        assert np.linalg.norm(r.x - ref.x) / np.linalg.norm(ref.x) <= 1e-12
        assert r.true_rel_residual == pytest.approx(ref.true_rel_residual, rel=1e-6)
    assert C.threads(1) == 1 and C.threads(0) >= 1


def test_c_oracle_edge_cases():
    """b = 0 gives x = 0 with no iteration; an iteration cap ends NOT_CONVERGED
    with the cap's iterate, the Python oracle's; an indefinite matrix breaks down."""
    from oracle import pcg_omp as C
    mesh = synth.box_mesh(6, 5, 4, 1, 1, 1)
    m, vals, A, dinv, _, _ = _system(mesh, 0.5)
    b = synth.uniform_vector(mesh, 0)
    r = C.pcg(m.row_ptr, m.col_idx, vals, dinv, np.zeros_like(b))
    assert r.status == O.OK and r.iterations == 0 and not r.x.any()
    r = C.pcg(m.row_ptr, m.col_idx, vals, dinv, b, tol=1e-12, max_iter=5)
    ref = O.pcg(A, dinv, b, tol=1e-12, max_iter=5)
    assert r.status == ref.status == O.NOT_CONVERGED and r.iterations == 5
    assert np.linalg.norm(r.x - ref.x) / np.linalg.norm(ref.x) <= 1e-13
    neg = -vals
    r = C.pcg(m.row_ptr, m.col_idx, neg, 1.0 / neg[m.diag_pos], b)
    ref = O.pcg(O.csr_matrix(m.row_ptr, m.col_idx, neg), 1.0 / neg[m.diag_pos], b)
    # D^-1 A is unchanged but p.Ap < 0 at once
    assert r.status == ref.status == O.BREAKDOWN and r.iterations == ref.iterations == 0


# ---------------------------------------------------------------- scaled inner system


def _scaled(mesh, sigma):
    m, vals, A, dinv, _, _ = _system(mesh, sigma)
    s = O.jacobi_scaling(vals[m.diag_pos])
    Ah32 = O.csr_matrix(m.row_ptr, m.col_idx, O.scaled_fp32_values(m.row_ptr, m.col_idx, vals, s))
    return m, vals, A, dinv, s, Ah32


def test_scaled_values_are_s_a_s():
    """fl32(a_ij s_i s_j) against the dense product S A S in FP64: within FP32
    rounding, a diagonal of exact ones, exactly symmetric; s_i^2 a_ii = 1 to
    FP64 rounding."""
    mesh = synth.box_mesh(7, 6, 5, 2, 1, 1)
    m, vals, A, dinv, s, Ah32 = _scaled(mesh, 1.0)
    d = A.diagonal()
    assert s.dtype == np.float64
    assert np.all(np.abs(s * s * d - 1.0) <= 4 * 2.0 ** -53)
    dense = (s[:, None] * A.toarray()) * s[None, :]
    got = Ah32.toarray().astype(np.float64)
    assert np.all(np.abs(got - dense) <= 2.0 ** -24 * np.abs(dense) * (1 + 1e-12) + 1e-300)
    assert np.array_equal(got, got.T)
    assert np.array_equal(np.diag(got), np.ones(mesh.n_cells))


def test_cg_on_scaled_system_is_jacobi_pcg():
    """CG without a preconditioner on S A S from S b, mapped back by S, is PCG on
    A with the preconditioner S^2 iterate for iterate (FP64 arithmetic, FP64
    scaled matrix): the equivalence the scaled inner solves rest on. S^2 is the
    Jacobi inverse D^-1 to FP64 rounding, so the iterates are Jacobi-PCG's."""
    mesh = synth.box_mesh(12, 10, 8, 2, 1, 1)
    m, vals, A, dinv, s, _ = _scaled(mesh, 1.0)
    b = synth.uniform_vector(mesh, 0)
    sd = s
    row = np.repeat(np.arange(mesh.n_cells), np.diff(m.row_ptr))
    Ah64 = O.csr_matrix(m.row_ptr, m.col_idx, vals * (sd[row] * sd[m.col_idx]))
    for k in (1, 2, 7, 20):
        y, it, st = O.pcg_fp32(Ah64, lambda v: v, sd * b, rel_tol=0.0, max_iter=k, dtype=np.float64)
        ref = O.pcg(A, sd * sd, b, tol=0.0, max_iter=k)
        assert it == k == ref.iterations
        assert np.linalg.norm(sd * y - ref.x) / np.linalg.norm(ref.x) <= 1e-12, k
        jac = O.pcg(A, dinv, b, tol=0.0, max_iter=k)
        assert np.linalg.norm(sd * y - jac.x) / np.linalg.norm(jac.x) <= 1e-11, k


def test_scaled_refinement_forms():
    """Both refinement forms with FP32 inner solves on the scaled system reach the
    FP64 residual 1e-9 with iteration counts within 5% of the Jacobi-preconditioned
    forms; the restarted form's last pass stops near the target; with an exact (FP64)
    inner solve the continued form reproduces plain PCG up to the rounding of its
    residual replacements."""
    mesh = synth.box_mesh(16, 16, 16, 2, 2, 2)
    m, vals, A, dinv, s, Ah32 = _scaled(mesh, 1.0)
    b = synth.uniform_vector(mesh, 0)
    v32 = O.to_fp32(vals)
    A32 = O.csr_matrix(m.row_ptr, m.col_idx, v32)
    d32 = np.float32(1) / v32[m.diag_pos]
    x = np.linalg.solve(A.toarray(), b)
    for scaled, plain in ((O.mixed_reliable_scaled(A, Ah32, s, b, tol=1e-9, delta=0.1),
                           O.mixed_reliable(A, A32, d32, b, tol=1e-9, delta=0.1)),
                          (O.mixed_ir_scaled(A, Ah32, s, b, tol=1e-9), O.mixed_ir(A, A32, d32, b, tol=1e-9))):
        assert scaled.status == O.OK
        assert np.linalg.norm(b - A @ scaled.x) / np.linalg.norm(b) <= 1e-9
        assert np.linalg.norm(scaled.x - x) / np.linalg.norm(x) < 1e-6
        assert abs(scaled.iterations - plain.iterations) <= 0.05 * plain.iterations + 2
    ir = O.mixed_ir_scaled(A, Ah32, s, b, tol=1e-9)
    assert 1e-10 <= ir.true_rel_residual <= 1e-9 and ir.outer_iterations >= 2
    sd = s
    row = np.repeat(np.arange(mesh.n_cells), np.diff(m.row_ptr))
    Ah64 = O.csr_matrix(m.row_ptr, m.col_idx, vals * (sd[row] * sd[m.col_idx]))
    ref = O.pcg(A, dinv, b, tol=1e-10)
    ex = O.mixed_reliable_scaled(A, Ah64, s, b, tol=1e-10, delta=0.1, dtype=np.float64)
    assert ex.status == O.OK
    assert abs(ex.iterations - ref.iterations) <= 2 + ex.outer_iterations // 2
    assert np.linalg.norm(ex.x - ref.x) / np.linalg.norm(ref.x) < 1e-8
