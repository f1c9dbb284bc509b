"""The sliced layout the PCG iteration multiplies with, against the oracle.

* Layout: decoded on the host (slice descriptors, offset tables, 8-bit index
  words, CSR positions), every real entry must name the oracle's column and
  CSR position, in the row's CSR order; padding must carry position -1 and
  the diagonal's offset 0; the table lists the slice's distinct offsets in
  first-appearance order (entry k, then lane). Bit-exact.
* Values after an update: sliced vals = oracle vals at each position (0 for
  padding), vals32 = their round-to-nearest float32. Bit-exact.
* rp_iter_spmv against the oracle product: FP64 within 1e-13 (|A||x|)_i per
  row; FP32 (FP32 values and vector, FP32 fused multiply-adds over L terms)
  within L * 2^-24 * (|A32||x32|)_i against the exact product of the same
  float32 inputs.
* The sliced and CSR layouts give bitwise-identical products and solves: the
  same entries are summed in the same order, and at these sizes both K1
  kernels run rows / 256 blocks, so every row lands on the same thread and
  (p, q) is reduced in the same order.
* Matrices the layout does not take (a row of more than 32 entries, slices
  with more than 256 distinct offsets) and n_parts > 1 run on CSR.
"""
import types

import numpy as np
import pytest
import torch

from oracle import repart_oracle as O
from paper_2510_08536_gb300 import build, repart, synth

from gpu_util import Case, check_layout

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    repart.load()
    torch.cuda.set_device(0)


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


# ------------------------------------------------------------------ inputs


def _single_rank(n, lower, upper):
    z = np.zeros(0, np.int32)
    return types.SimpleNamespace(n_cells=n, lower_addr=np.asarray(lower, np.int32),
                                 upper_addr=np.asarray(upper, np.int32), iface_row=z, iface_nbr_rank=z,
                                 iface_nbr_col=z)


def _spd_staging(rank, seed):
    """[diag | upper | lower] of one rank: off-diagonals -a_f, diag = sum a_f + 1."""
    rng = np.random.default_rng(seed)
    a = rng.lognormal(0.0, 0.5, rank.lower_addr.shape[0])
    diag = np.ones(rank.n_cells)
    np.add.at(diag, rank.lower_addr, a)
    np.add.at(diag, rank.upper_addr, a)
    return np.concatenate([diag, -a, -a])


def _faces_from_pairs(pairs):
    pairs = np.unique(np.sort(np.asarray(pairs, np.int64), axis=1), axis=0)
    pairs = pairs[pairs[:, 0] != pairs[:, 1]]
    return pairs[:, 0], pairs[:, 1]


def _scrambled_box(nx, ny, nz, seed):
    """7-point box mesh, one rank, cells numbered at random (up to 224 offsets a slice)."""
    m = synth.box_mesh(nx, ny, nz, 1, 1, 1)
    r = m.ranks[0]
    perm = np.random.default_rng(seed).permutation(r.n_cells)
    lo, up = _faces_from_pairs(np.stack([perm[r.lower_addr], perm[r.upper_addr]], 1))
    return _single_rank(r.n_cells, lo, up)


def _banded(n, offsets):
    """Cell i coupled to i + d for each d: rows of up to 2 len(offsets) + 1 entries."""
    pairs = [(i, i + d) for d in offsets for i in range(n - d)]
    lo, up = _faces_from_pairs(pairs)
    return _single_rank(n, lo, up)


class Sys:
    """A matrix given as rank descriptors + staging, with its oracle map and values."""

    def __init__(self, ranks, staging, seed=0):
        self.ranks = ranks
        self.staging = staging
        (self.map,) = O.repartition_map(ranks, 1)
        self.vals = O.update_values(self.map.src_of, staging)
        self.n = int(self.map.row_ptr.shape[0] - 1)
        self.A = O.csr_matrix(self.map.row_ptr, self.map.col_idx, self.vals)
        self.b = np.random.default_rng(seed).uniform(-1.0, 1.0, self.n)


def _box(dims, parts, sigma=0.5):
    c = Case(dims, parts, sigma=sigma, oracle_map=False)
    return Sys(c.mesh.ranks, c.staging)


def _custom(rank, seed=5):
    return Sys([rank], _spd_staging(rank, seed))


SYSTEMS = {
    "box32_k8": lambda: _box((32, 32, 32), (2, 2, 2)),
    "box13x7x9_k6": lambda: _box((13, 7, 9), (3, 2, 1)),
    "slab40_k4": lambda: _box((40, 3, 2), (4, 1, 1)),
    "two_cells": lambda: _box((2, 1, 1), (2, 1, 1)),
    "scrambled_9x8x7": lambda: _custom(_scrambled_box(9, 8, 7, 3)),
    "banded_wide": lambda: _custom(_banded(1500, [1, 2, 3, 5, 8, 13, 21, 34, 55, 89, 144, 233])),
}


# ------------------------------------------------------------------ tests


@pytest.mark.parametrize("name", list(SYSTEMS))
def test_layout_and_values_bit_exact(name):
    S = SYSTEMS[name]()
    h = repart.build_repartition(S.ranks)
    repart.update_values_packed(h, _t(S.staging))
    view = repart.get_sliced_view(h)
    assert view is not None, "layout not built"
    check_layout(view, S.map, S.n)
    # the uniform-slice flag: every slice 4-bit (table reference bit 31) with rows
    # of at most 8 entries -- the iteration then runs the kernel instance without
    # the general case's checks (the parity tests below cover both instances)
    d = view["desc"].cpu().numpy().view(np.uint32).reshape(-1, 2)[: view["n_slices"] + 1, 0].astype(np.int64)
    w4 = (view["tinfo"].cpu().numpy().view(np.uint32) >> 31) == 1
    expect = bool(w4.all() and (np.diff(d) // 32 <= 8).all())
    assert view["uniform4"] == expect, (name, view["uniform4"], expect)
    if name == "box32_k8":  # 7-point stencil, equal cubic ranks: few offsets a slice
        assert view["uniform4"]
    if name == "banded_wide":  # rows of up to 25 entries
        assert not view["uniform4"]
    pos = view["pos"].cpu().numpy()
    want = np.where(pos >= 0, S.vals[np.maximum(pos, 0)], 0.0)
    np.testing.assert_array_equal(view["vals"].cpu().numpy(), want)
    np.testing.assert_array_equal(view["vals32"].cpu().numpy(), want.astype(np.float32))
    h.close()


@pytest.mark.parametrize("name", list(SYSTEMS))
def test_iter_spmv_parity(name):
    S = SYSTEMS[name]()
    h = repart.build_repartition(S.ranks)
    repart.update_values_packed(h, _t(S.staging))
    assert repart.get_sliced_view(h) is not None
    rng = np.random.default_rng(11)
    x = rng.uniform(-1.0, 1.0, S.n)
    absA = abs(S.A)
    # FP64
    y = torch.empty(S.n, dtype=torch.float64, device=DEV)
    repart.iter_spmv(h, _t(x), y, "fp64")
    ref = O.spmv(S.map.row_ptr, S.map.col_idx, S.vals, x)
    bound = 1e-13 * (absA @ np.abs(x))
    assert (np.abs(y.cpu().numpy() - ref) <= bound).all()
    # FP32: exact product of the float32 inputs, FP32 accumulation bound
    x32 = x.astype(np.float32)
    y32 = torch.empty(S.n, dtype=torch.float32, device=DEV)
    repart.iter_spmv(h, _t(x32), y32, "mixed")
    v32 = O.to_fp32(S.vals).astype(np.float64)
    ref32 = O.spmv(S.map.row_ptr, S.map.col_idx, v32, x32.astype(np.float64))
    L = np.diff(S.map.row_ptr).max()
    bound32 = L * 2.0 ** -24 * (O.csr_matrix(S.map.row_ptr, S.map.col_idx, np.abs(v32)) @ np.abs(x32.astype(np.float64)))
    assert (np.abs(y32.cpu().numpy().astype(np.float64) - ref32) <= bound32 * 1.0001 + 1e-30).all()
    h.close()


@pytest.mark.parametrize("name", ["box32_k8", "scrambled_9x8x7", "banded_wide"])
def test_sliced_and_csr_layouts_agree_bitwise(name):
    S = SYSTEMS[name]()
    hs = repart.build_repartition(S.ranks)
    hc = repart.build_repartition(S.ranks, layout=repart.RP_LAYOUT_CSR)
    assert repart.get_sliced_view(hs) is not None and repart.get_sliced_view(hc) is None
    for h in (hs, hc):
        repart.update_values_packed(h, _t(S.staging))
    x = _t(np.random.default_rng(2).uniform(-1.0, 1.0, S.n))
    ys = [torch.empty_like(x) for _ in range(2)]
    for h, y in zip((hs, hc), ys):
        repart.iter_spmv(h, x, y, "fp64")
    assert torch.equal(ys[0], ys[1])
    x32 = x.float()
    ys = [torch.empty_like(x32) for _ in range(2)]
    for h, y in zip((hs, hc), ys):
        repart.iter_spmv(h, x32, y, "mixed")
    assert torch.equal(ys[0], ys[1])
    b = _t(S.b)
    for precision in ("fp64", "mixed", "mixed_ru"):
        xs = [torch.zeros(S.n, dtype=torch.float64, device=DEV) for _ in range(2)]
        infos = [repart.solve(h, b, xx, tol=1e-9, precision=precision) for h, xx in zip((hs, hc), xs)]
        assert infos[0]["status"] == infos[1]["status"] == 0
        for xx in xs:
            assert np.linalg.norm(S.b - S.A @ xx.cpu().numpy()) / np.linalg.norm(S.b) <= 1e-9
        if precision == "fp64":
            assert infos[0] == infos[1], (precision, infos)
            assert torch.equal(xs[0], xs[1]), precision
        else:
            # the sliced handle's inner iteration runs on S A S (Jacobi made explicit),
            # the CSR one Jacobi-preconditioned on A: each against its oracle form
            # (equal in exact arithmetic, FP32 rounding differs)
            s_ = O.jacobi_scaling(S.vals[S.map.diag_pos])
            Ah = O.csr_matrix(S.map.row_ptr, S.map.col_idx,
                              O.scaled_fp32_values(S.map.row_ptr, S.map.col_idx, S.vals, s_))
            v32 = O.to_fp32(S.vals)
            A32 = O.csr_matrix(S.map.row_ptr, S.map.col_idx, v32)
            d32 = np.float32(1) / v32[S.map.diag_pos]
            if precision == "mixed":
                refs = (O.mixed_ir_scaled(S.A, Ah, s_, S.b, tol=1e-9), O.mixed_ir(S.A, A32, d32, S.b, tol=1e-9))
            else:
                refs = (O.mixed_reliable_scaled(S.A, Ah, s_, S.b, tol=1e-9, delta=0.1),
                        O.mixed_reliable(S.A, A32, d32, S.b, tol=1e-9, delta=0.1))
            fp64 = O.pcg(S.A, O.jacobi_inverse(S.map.row_ptr, S.map.col_idx, S.vals, S.map.diag_pos), S.b,
                         tol=1e-9).iterations
            for inf, ref in zip(infos, refs):
                # rounding order differs from the oracle's: see test_gpu_parity._inner_count_ok
                assert 0.95 * fp64 - 5 <= inf["iterations"] <= 1.10 * ref.iterations + 10, (precision, infos,
                                                                                            ref.iterations, fp64)
    hs.close()
    hc.close()


@pytest.mark.parametrize("name", ["box32_k8", "scrambled_9x8x7"])
def test_scaled_inner_values_bit_exact(name):
    """After a mixed solve the FP32 sliced values of S A S and the scaling s equal
    the oracle's (jacobi_scaling, scaled_fp32_values) bit for bit, padding 0; a
    value update refills them from the new values."""
    S = SYSTEMS[name]()
    h = repart.build_repartition(S.ranks)
    repart.update_values_packed(h, _t(S.staging))
    assert repart.get_sliced_view(h)["vals32s"] is None  # made by the first mixed solve
    x = torch.zeros(S.n, dtype=torch.float64, device=DEV)
    assert repart.solve(h, _t(S.b), x, tol=1e-9, precision="mixed_ru")["status"] == 0
    for staging in (S.staging, 1.5 * S.staging):
        repart.update_values_packed(h, _t(staging))
        vals = O.update_values(S.map.src_of, staging)
        view = repart.get_sliced_view(h)
        s = O.jacobi_scaling(vals[S.map.diag_pos])
        np.testing.assert_array_equal(view["scale"].cpu().numpy(), s)
        want = O.scaled_fp32_values(S.map.row_ptr, S.map.col_idx, vals, s)
        pos = view["pos"].cpu().numpy()
        exp = np.where(pos >= 0, want[np.maximum(pos, 0)], np.float32(0))
        np.testing.assert_array_equal(view["vals32s"].cpu().numpy(), exp)
    h.close()


def _hub(n=200, fan=40):
    """A chain plus one cell coupled to `fan` others: a row of fan + 2 entries."""
    pairs = [(i, i + 1) for i in range(n - 1)] + [(0, j) for j in range(2, 2 + fan)]
    lo, up = _faces_from_pairs(pairs)
    return _single_rank(n, lo, up)


def _random_graph(n=640, deg=10, seed=4):
    """Random couplings: ~20 off-diagonals a row at unrelated offsets (> 256 per slice)."""
    rng = np.random.default_rng(seed)
    pairs = np.stack([np.repeat(np.arange(n), deg), rng.integers(0, n, n * deg)], 1)
    lo, up = _faces_from_pairs(pairs)
    return _single_rank(n, lo, up)


@pytest.mark.parametrize("make", [_hub, _random_graph])
def test_layout_falls_back_to_csr(make):
    S = _custom(make())
    h = repart.build_repartition(S.ranks)
    assert repart.get_sliced_view(h) is None
    repart.update_values_packed(h, _t(S.staging))
    x = _t(np.random.default_rng(1).uniform(-1.0, 1.0, S.n))
    y = torch.empty_like(x)
    repart.iter_spmv(h, x, y, "fp64")
    ref = O.spmv(S.map.row_ptr, S.map.col_idx, S.vals, x.cpu().numpy())
    assert (np.abs(y.cpu().numpy() - ref) <= 1e-13 * (abs(S.A) @ np.abs(x.cpu().numpy()))).all()
    xs = torch.zeros(S.n, dtype=torch.float64, device=DEV)
    info = repart.solve(h, _t(S.b), xs, tol=1e-9)
    assert info["status"] == 0
    assert np.linalg.norm(S.b - S.A @ xs.cpu().numpy()) / np.linalg.norm(S.b) <= 1e-9
    h.close()


@pytest.mark.parametrize("dims,parts,n_parts", [((12, 10, 8), (2, 2, 1), 2), ((13, 7, 9), (3, 2, 1), 3),
                                                 ((13, 7, 9), (3, 2, 1), 6), ((40, 3, 2), (4, 1, 1), 4)])
def test_multi_part_sliced(dims, parts, n_parts):
    """Several GPU parts: each part's rows in slices of their own (ragged part
    ends), local entries in the slices, non-local entries after them -- the
    same row sums as the CSR iteration bit for bit, solves as the oracle's."""
    c = Case(dims, parts, oracle_map=False)
    h = repart.build_repartition(c.mesh.ranks, n_parts=n_parts)
    hc = repart.build_repartition(c.mesh.ranks, n_parts=n_parts, layout=repart.RP_LAYOUT_CSR)
    assert repart.get_sliced_view(hc) is None
    for hh in (h, hc):
        repart.update_values_packed(hh, _t(c.staging))
    view = repart.get_sliced_view(h)
    assert view is not None, "layout not built"
    maps = O.repartition_map(c.mesh.ranks, n_parts)
    srow = view["srow"].cpu().numpy().reshape(-1, 2)
    desc = view["desc"].cpu().numpy().view(np.uint32).reshape(-1, 2).astype(np.int64)
    pos = view["pos"].cpu().numpy().astype(np.int64)
    vals = repart.get_values(h)["vals"].cpu().numpy()
    s0 = r0 = nnz0 = 0
    for p, m in enumerate(maps):
        n_p = m.row_ptr.shape[0] - 1
        S_p = (n_p + 31) // 32
        np.testing.assert_array_equal(srow[s0:s0 + S_p, 0], r0 + 32 * np.arange(S_p))
        np.testing.assert_array_equal(srow[s0:s0 + S_p, 1] >> 6, p)
        np.testing.assert_array_equal(srow[s0:s0 + S_p, 1] & 63, np.minimum(32, n_p - 32 * np.arange(S_p)))
        e0, e1 = desc[s0, 0], desc[s0 + S_p, 0]
        local = np.where(pos >= 0, pos - nnz0, -1)
        sub = dict(view, n_slices=S_p, n_entries=int(e1 - e0), desc=view["desc"][2 * s0:2 * (s0 + S_p + 1)],
                   tinfo=view["tinfo"][s0:s0 + S_p], pos=torch.from_numpy(local))
        check_layout(sub, m, n_p)
        lp = pos[e0:e1]
        np.testing.assert_array_equal(view["vals"].cpu().numpy()[e0:e1], np.where(lp >= 0, vals[np.maximum(lp, 0)], 0.0))
        s0 += S_p
        r0 += n_p
        nnz0 += m.col_idx.shape[0]
    assert s0 == view["n_slices"]
    # products: bitwise those of the CSR iteration
    n = c.mesh.n_cells
    x = _t(np.random.default_rng(2).uniform(-1.0, 1.0, n))
    ys = [torch.empty_like(x) for _ in range(2)]
    for hh, y in zip((h, hc), ys):
        repart.iter_spmv(hh, x, y, "fp64")
    assert torch.equal(ys[0], ys[1])
    x32 = x.float()
    ys = [torch.empty_like(x32) for _ in range(2)]
    for hh, y in zip((h, hc), ys):
        repart.iter_spmv(hh, x32, y, "mixed")
    assert torch.equal(ys[0], ys[1])
    # solves: the oracle's system, all three precisions
    (m1,) = O.repartition_map(c.mesh.ranks, 1)
    A = O.csr_matrix(m1.row_ptr, m1.col_idx, O.update_values(m1.src_of, c.staging))
    dinv = O.jacobi_inverse(m1.row_ptr, m1.col_idx, O.update_values(m1.src_of, c.staging), m1.diag_pos)
    ref = O.pcg(A, dinv, c.b, tol=1e-9)
    for precision in ("fp64", "mixed", "mixed_ru"):
        xs = torch.zeros(n, dtype=torch.float64, device=DEV)
        info = repart.solve(h, _t(c.b), xs, tol=1e-9, precision=precision)
        xn = xs.cpu().numpy()
        assert info["status"] == 0, (precision, info)
        assert np.linalg.norm(c.b - A @ xn) / np.linalg.norm(c.b) <= 1e-9, precision
        if precision == "fp64":
            assert np.linalg.norm(xn - ref.x) / np.linalg.norm(ref.x) <= 1e-7
            assert abs(info["iterations"] - ref.iterations) <= 2
    h.close()
    hc.close()


def test_adjoint_on_sliced_layout_bitwise():
    """The adjoint of general storage multiplies with the sliced layout filled
    from the transposed values: the same lambda, bit for bit, as on CSR."""
    c = Case((16, 12, 10), (2, 2, 2), sigma=0.5, oracle_map=False)
    n = c.mesh.n_cells
    lams = []
    for layout in (repart.RP_LAYOUT_AUTO, repart.RP_LAYOUT_CSR):
        h = repart.build_repartition(c.mesh.ranks, want_transpose=True, layout=layout)
        assert (repart.get_sliced_view(h) is not None) == (layout == repart.RP_LAYOUT_AUTO)
        repart.update_values_packed(h, _t(c.staging))
        x = torch.zeros(n, dtype=torch.float64, device=DEV)
        repart.solve(h, _t(c.b), x, tol=1e-12)
        g = x - _t(synth.uniform_vector(c.mesh, 1))
        lam = torch.zeros_like(x)
        info = repart.solve_adjoint(h, g, lam, tol=1e-12)
        assert info["status"] == 0
        lams.append((lam, info))
        h.close()
    assert lams[0][1] == lams[1][1]
    assert torch.equal(lams[0][0], lams[1][0])
