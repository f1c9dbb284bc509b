"""CPU oracle of the repartitioning hot path.

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import, call or
execute this module: only the tests, the smoke check of ``__graft_entry__``
and the CPU-baseline / reference leg of ``bench.py`` use it. It shares no
code with the CUDA path; it reads its inputs (rank descriptors, staging
buffers, right-hand sides) as plain arrays.

Everything is plain NumPy in FP64 (FP32 only where the mixed form says so),
written for a reader to check against the paper by eye:

* blockwise ownership of CPU ranks by GPU parts, ``n_GPU = n_CPU / alpha``
  (Sec. 3);
* the local / non-local split of coefficients and the localisation of
  interface entries whose column lies in the part's own rows, the criterion
  ``j in I_GPU(r) = union_l I_CPU(alpha*r + l)`` (Sec. 3, steps 1-3);
* the three outputs of the repartitioning: sparsity pattern, update pattern
  (per-rank offsets into one continuous buffer) and the permutation from LDU
  order to row-major order (Sec. 3);
* the value update: the continuous buffer reordered by that permutation
  (Sec. 3, update procedure);
* Jacobi-preconditioned CG for the merged pressure system (the paper solves
  it with CG, Sec. 4; the preconditioner is Jacobi here);
* Jacobi-preconditioned BiCGStab for the non-symmetric momentum system (the
  paper's momentum solver, Sec. 4), in FP64 and as FP32-inner / FP64-outer
  refinement;
* FP32-inner / FP64-outer iterative refinement, the adjoint solve and the
  gradients with respect to the stored entries (plain definitions).

Library primitives used as single steps: ``numpy.lexsort`` (sorting) and
``scipy.sparse.csr_matrix @ x`` (a sparse matrix-vector product).

Pins: every function is checked in ``tests/test_oracle_pins.py`` against
hand-enumerated maps, ``scipy.sparse`` COO->CSR conversion, dense solves,
the closed-form eigenpairs of the 7-point operator, a face-loop LDU product
written independently below, decomposition invariance and central finite
differences.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp

# --------------------------------------------------------------------------
# Ownership and layout (Sec. 3, blockwise distribution)
# --------------------------------------------------------------------------


def rank_offsets(ranks) -> np.ndarray:
    """off[r] = first merged row of CPU rank r; off[k] = total rows.

    Under blockwise ownership the merged numbering of a part is the
    concatenation of its ranks' local numberings (Sec. 3)."""
    off = np.zeros(len(ranks) + 1, np.int64)
    for r, d in enumerate(ranks):
        off[r + 1] = off[r] + int(d.n_cells)
    return off


def slot_offsets(ranks, symmetric: bool) -> np.ndarray:
    """Start of each rank's block in the continuous coefficient buffer.

    Each rank contributes ``[diag n | upper F | lower F | iface E]`` (no
    ``lower`` when the matrix is symmetric): the buffer is ordered by rank,
    then by LDU order (Sec. 3, update procedure)."""
    off = np.zeros(len(ranks) + 1, np.int64)
    for r, d in enumerate(ranks):
        f = len(d.lower_addr)
        off[r + 1] = off[r] + int(d.n_cells) + (1 if symmetric else 2) * f + len(d.iface_row)
    return off


def part_of_rank(k: int, n_parts: int) -> np.ndarray:
    """GPU part of every CPU rank: part p owns ranks alpha*p .. alpha*p+alpha-1
    with alpha = k / n_parts (Sec. 3)."""
    if n_parts < 1 or k % n_parts:
        raise ValueError("n_parts must divide the number of CPU ranks")
    alpha = k // n_parts
    return np.arange(k, dtype=np.int64) // alpha


def coo_entries(ranks, symmetric: bool):
    """Every stored coefficient as (global row, global col, buffer slot).

    Step 1 of Sec. 3: the sparsity pattern of each LDU matrix including its
    coupling to non-local entries. Entry conventions: diag (i, i); upper[f]
    at (l_f, u_f); lower[f] at (u_f, l_f); interface entry e at
    (row_e, col_e of rank q_e). In symmetric mode the lower triangle reads
    the upper slot."""
    off = rank_offsets(ranks)
    soff = slot_offsets(ranks, symmetric)
    rows, cols, slots = [], [], []
    for r, d in enumerate(ranks):
        n = int(d.n_cells)
        lo = np.asarray(d.lower_addr, np.int64)
        up = np.asarray(d.upper_addr, np.int64)
        f = lo.shape[0]
        ir = np.asarray(d.iface_row, np.int64)
        iq = np.asarray(d.iface_nbr_rank, np.int64)
        ic = np.asarray(d.iface_nbr_col, np.int64)
        s0 = soff[r]
        i = np.arange(n, dtype=np.int64)
        rows += [off[r] + i, off[r] + lo, off[r] + up]
        cols += [off[r] + i, off[r] + up, off[r] + lo]
        upper_slot = s0 + n + np.arange(f, dtype=np.int64)
        lower_slot = upper_slot if symmetric else s0 + n + f + np.arange(f, dtype=np.int64)
        iface_slot = s0 + n + (1 if symmetric else 2) * f + np.arange(ir.shape[0], dtype=np.int64)
        slots += [s0 + i, upper_slot, lower_slot]
        rows.append(off[r] + ir)
        cols.append(off[iq] + ic)
        slots.append(iface_slot)
    return np.concatenate(rows), np.concatenate(cols), np.concatenate(slots)


def row_entries(ranks, row: int, symmetric: bool = False):
    """The stored entries of one merged row, straight from the definitions:
    sorted (global col, buffer slot) pairs. Slow; for sampling large maps."""
    off = rank_offsets(ranks)
    soff = slot_offsets(ranks, symmetric)
    r = int(np.searchsorted(off, row, side="right") - 1)
    d = ranks[r]
    i = row - int(off[r])
    n = int(d.n_cells)
    lo = np.asarray(d.lower_addr, np.int64)
    up = np.asarray(d.upper_addr, np.int64)
    f = lo.shape[0]
    s0 = int(soff[r])
    out = [(row, s0 + i)]
    for fi in np.nonzero(lo == i)[0]:
        out.append((int(off[r] + up[fi]), s0 + n + int(fi)))
    for fi in np.nonzero(up == i)[0]:
        out.append((int(off[r] + lo[fi]), s0 + n + int(fi) + (0 if symmetric else f)))
    base = s0 + n + (1 if symmetric else 2) * f
    ir = np.asarray(d.iface_row, np.int64)
    for e in np.nonzero(ir == i)[0]:
        q = int(d.iface_nbr_rank[e])
        out.append((int(off[q] + d.iface_nbr_col[e]), base + int(e)))
    return sorted(out)


def _csr(rows, cols, slots, n_rows):
    """Row-major ordering with ascending columns inside a row."""
    order = np.lexsort((cols, rows))
    r, c, s = rows[order], cols[order], slots[order]
    if r.shape[0] > 1:
        dup = (r[1:] == r[:-1]) & (c[1:] == c[:-1])
        if dup.any():
            raise ValueError("duplicate (row, col) entry")
    row_ptr = np.zeros(n_rows + 1, np.int64)
    np.cumsum(np.bincount(r, minlength=n_rows), out=row_ptr[1:])
    return row_ptr, c, s


@dataclasses.dataclass
class PartMap:
    """The repartitioned matrix of one GPU part (Sec. 3, three outputs)."""

    row_off: int            # first merged row of the part
    n_rows: int
    buf_off: int            # start of the part's slice of the continuous buffer
    buf_len: int
    row_ptr: np.ndarray     # local CSR
    col_idx: np.ndarray     # part-local columns
    src_of: np.ndarray      # permutation: buffer slot feeding CSR position p
    diag_pos: np.ndarray
    tpos: np.ndarray        # CSR position of the transposed entry
    nl_row_ptr: np.ndarray  # non-local CSR (rows of the part)
    nl_col_idx: np.ndarray  # compressed non-local column
    nl_src_of: np.ndarray
    nl_cols: np.ndarray     # global column of each compressed non-local column


def repartition_map(ranks, n_parts: int = 1, symmetric: bool = False):
    """Fuse the sparsity patterns of the CPU ranks into one pattern per GPU part.

    Sec. 3, step 3: a part fuses the local patterns of its alpha ranks; an
    interface entry joins the local pattern when its column lies in the
    part's rows, otherwise the non-local pattern, whose columns are the
    ascending list of distinct remote global columns. Returns one PartMap
    per part; ``src_of`` indexes the part's own slice of the buffer."""
    k = len(ranks)
    part = part_of_rank(k, n_parts)
    off = rank_offsets(ranks)
    soff = slot_offsets(ranks, symmetric)
    rows, cols, slots = coo_entries(ranks, symmetric)
    alpha = k // n_parts
    out = []
    for p in range(n_parts):
        r0, r1 = off[p * alpha], off[(p + 1) * alpha]
        b0, b1 = soff[p * alpha], soff[(p + 1) * alpha]
        mine = (rows >= r0) & (rows < r1)
        local = mine & (cols >= r0) & (cols < r1)       # j in I_GPU(p)
        remote = mine & ~local
        n_rows = int(r1 - r0)
        row_ptr, col_idx, src_of = _csr(rows[local] - r0, cols[local] - r0, slots[local] - b0, n_rows)
        # diagonal position and transposed position of each entry
        row_of = np.repeat(np.arange(n_rows, dtype=np.int64), np.diff(row_ptr))
        diag_pos = np.full(n_rows, -1, np.int64)
        is_d = row_of == col_idx
        diag_pos[row_of[is_d]] = np.nonzero(is_d)[0]
        key = row_of * n_rows + col_idx                    # sorted ascending
        tkey = col_idx * n_rows + row_of
        tpos = np.searchsorted(key, tkey)
        tpos_ok = (tpos < key.shape[0]) & (key[np.minimum(tpos, key.shape[0] - 1)] == tkey)
        tpos = np.where(tpos_ok, tpos, -1)
        nl_cols = np.unique(cols[remote])
        nl_row_ptr, nl_col_idx, nl_src_of = _csr(
            rows[remote] - r0, np.searchsorted(nl_cols, cols[remote]), slots[remote] - b0, n_rows)
        out.append(PartMap(int(r0), n_rows, int(b0), int(b1 - b0), row_ptr, col_idx, src_of,
                           diag_pos, tpos, nl_row_ptr, nl_col_idx, nl_src_of, nl_cols))
    return out


# --------------------------------------------------------------------------
# Value update (Sec. 3, update procedure)
# --------------------------------------------------------------------------


def pack_buffer(rank_arrays, symmetric: bool) -> np.ndarray:
    """The continuous buffer: per rank diag, upper, (lower,) iface, in rank order."""
    parts = []
    for diag, upper, lower, iface in rank_arrays:
        parts += [np.asarray(diag, np.float64), np.asarray(upper, np.float64)]
        if not symmetric:
            parts.append(np.asarray(lower, np.float64))
        parts.append(np.asarray(iface, np.float64))
    return np.concatenate(parts) if parts else np.zeros(0)


def update_values(src_of: np.ndarray, buffer: np.ndarray) -> np.ndarray:
    """vals[p] = buffer[src_of[p]]: the buffer reordered by the permutation."""
    return buffer[src_of]


def to_fp32(vals: np.ndarray) -> np.ndarray:
    """FP32 copy of the values, round to nearest even."""
    return vals.astype(np.float32)


# --------------------------------------------------------------------------
# Matrix-vector products
# --------------------------------------------------------------------------


def csr_matrix(row_ptr, col_idx, vals, n_cols=None):
    n = row_ptr.shape[0] - 1
    return sp.csr_matrix((vals, col_idx, row_ptr), shape=(n, n if n_cols is None else n_cols))


def spmv(row_ptr, col_idx, vals, x):
    """y_i = sum over stored (i, j) of a_ij x_j."""
    return csr_matrix(row_ptr, col_idx, vals, x.shape[0]) @ x


def ldu_matvec(ranks, buffer, x, symmetric: bool = False):
    """Sum over CPU ranks of the LDU product plus interface coupling.

    Written face by face, the way an LDU matrix is applied (rank r, face f:
    y[l] += upper[f] x[u], y[u] += lower[f] x[l]), with no repartitioning at
    all; its result must equal the merged CSR product."""
    off = rank_offsets(ranks)
    soff = slot_offsets(ranks, symmetric)
    y = np.zeros(int(off[-1]), np.float64)
    for r, d in enumerate(ranks):
        n = int(d.n_cells)
        lo = np.asarray(d.lower_addr, np.int64) + off[r]
        up = np.asarray(d.upper_addr, np.int64) + off[r]
        f = lo.shape[0]
        s = int(soff[r])
        diag = buffer[s:s + n]
        upper = buffer[s + n:s + n + f]
        lower = upper if symmetric else buffer[s + n + f:s + n + 2 * f]
        iface = buffer[s + n + (1 if symmetric else 2) * f:int(soff[r + 1])]
        rows = slice(int(off[r]), int(off[r + 1]))
        y[rows] += diag * x[rows]
        np.add.at(y, lo, upper * x[up])
        np.add.at(y, up, lower * x[lo])
        gcol = off[np.asarray(d.iface_nbr_rank, np.int64)] + np.asarray(d.iface_nbr_col, np.int64)
        np.add.at(y, off[r] + np.asarray(d.iface_row, np.int64), iface * x[gcol])
    return y


# --------------------------------------------------------------------------
# Jacobi-preconditioned CG (textbook PCG)
# --------------------------------------------------------------------------

OK, NOT_CONVERGED, BREAKDOWN = 0, 7, 8


@dataclasses.dataclass
class SolveResult:
    x: np.ndarray
    iterations: int
    status: int
    rel_residual: float       # recursive residual at exit
    true_rel_residual: float  # ||b - A x|| / ||b|| recomputed at exit
    outer_iterations: int = 0


def jacobi_inverse(row_ptr, col_idx, vals, diag_pos=None):
    """1 / a_ii (FP64, correctly rounded division)."""
    if diag_pos is None:
        n = row_ptr.shape[0] - 1
        row_of = np.repeat(np.arange(n), np.diff(row_ptr))
        diag = np.zeros(n, vals.dtype)
        m = row_of == col_idx
        diag[row_of[m]] = vals[m]
    else:
        diag = vals[diag_pos]
    one = np.array(1.0, diag.dtype)
    return one / diag


def _operator(prec):
    """A preconditioner as z = prec(r): an array is the Jacobi inverse diagonal."""
    if callable(prec):
        return prec
    return lambda r: prec * r


def line_part(row_ptr, col_idx, vals, block=32):
    """The line (block-tridiagonal) part M of a matrix: per row i its diagonal and
    the couplings (i, i-1) and (i, i+1) that stay inside i's block of ``block``
    consecutive rows (blocks start at multiples of ``block``). Returns
    (sub, diag, sup): sub[i] = A[i, i-1] (0 at a block start), sup[i] = A[i, i+1]
    (0 at a block end). On a line-ordered mesh (rows x-fastest, x-lines of
    ``block`` cells) M is the x-line part of A: block-Jacobi over the lines."""
    n = row_ptr.shape[0] - 1
    row = np.repeat(np.arange(n), np.diff(row_ptr))
    col = np.asarray(col_idx, np.int64)
    sub = np.zeros(n, vals.dtype)
    diag = np.zeros(n, vals.dtype)
    sup = np.zeros(n, vals.dtype)
    m = col == row
    diag[row[m]] = vals[m]
    m = (col == row - 1) & (row % block != 0)
    sub[row[m]] = vals[m]
    m = (col == row + 1) & (row % block != block - 1)
    sup[row[m]] = vals[m]
    return sub, diag, sup


def line_operator(sub, diag, sup, dtype=np.float64):
    """z = M^-1 r for M = tridiag(sub, diag, sup), by one banded LU solve
    (scipy.linalg.solve_banded) in ``dtype``; the zero couplings at block
    boundaries make it independent solves per block."""
    import scipy.linalg as sla
    n = diag.shape[0]
    ab = np.zeros((3, n), dtype)
    ab[0, 1:] = sup[:-1]
    ab[1] = diag
    ab[2, :-1] = sub[1:]
    return lambda r: sla.solve_banded((1, 1), ab, np.asarray(r, dtype))


def pcg(A, dinv, b, tol=1e-9, max_iter=10000, x0=None) -> SolveResult:
    """Preconditioned CG with z = D^-1 r.

    x0 = 0 unless given; r = b - A x; z = D^-1 r; p = z; per iteration
    alpha = (r.z)/(p.Ap), x += alpha p, r -= alpha Ap; stop when
    ||r|| <= tol ||b||, after confirming with the true residual b - A x (if
    that fails, r is replaced by it and the iteration restarts from p = z);
    otherwise z = D^-1 r, beta = (r.z)_new/(r.z)_old, p = z + beta p.
    ``dinv`` is the Jacobi inverse diagonal, or any preconditioner z = dinv(r)."""
    prec = _operator(dinv)
    b = np.asarray(b, np.float64)
    bb = float(b @ b)
    if bb == 0.0:
        return SolveResult(np.zeros_like(b), 0, OK, 0.0, 0.0)
    thresh = tol * tol * bb
    x = np.zeros_like(b) if x0 is None else np.array(x0, np.float64)
    r = b - A @ x if x0 is not None else b.copy()
    it = 0
    status = NOT_CONVERGED
    rr = float(r @ r)
    restart = True
    while True:
        if restart:
            z = prec(r)
            p = z.copy()
            rz = float(r @ z)
            restart = False
            if rr <= thresh:
                tr = b - A @ x
                if float(tr @ tr) <= thresh:
                    status = OK
                    break
        if it >= max_iter:
            break
        q = A @ p
        pq = float(p @ q)
        if not pq > 0.0:
            status = BREAKDOWN
            break
        alpha = rz / pq
        x += alpha * p
        r -= alpha * q
        it += 1
        rr = float(r @ r)
        if rr <= thresh:
            tr = b - A @ x
            trr = float(tr @ tr)
            if trr <= thresh:
                status = OK
                break
            r = tr
            rr = trr
            restart = True
            continue
        z = prec(r)
        rz_new = float(r @ z)
        beta = rz_new / rz
        p = z + beta * p
        rz = rz_new
    tr = b - A @ x
    return SolveResult(x, it, status, float(np.sqrt(rr / bb)), float(np.sqrt((tr @ tr) / bb)))


def bicgstab(A, dinv, b, tol=1e-9, max_iter=10000, x0=None) -> SolveResult:
    """Jacobi-preconditioned BiCGStab (van der Vorst, 1992) for the non-symmetric
    momentum system (the paper's momentum solver is BiCGStab, Sec. 4), with the
    preconditioner applied to the search directions (right preconditioning).

    From r = b - A x (x0 = 0 unless given) and the shadow residual rhat = r, with
    rho_old = alpha = omega = 1 and p = v = 0, each iteration takes
    rho = (rhat, r), beta = (rho / rho_old)(alpha / omega), p = r + beta (p - omega v),
    phat = D^-1 p, v = A phat, alpha = rho / (rhat, v), s = r - alpha v; if
    ||s|| <= tol ||b|| it ends with x += alpha phat; else shat = D^-1 s, t = A shat,
    omega = (t, s) / (t, t), x += alpha phat + omega shat, r = s - omega t. Each
    iteration counts once (two products with A). A recursive residual at the target
    is confirmed with b - A x; if that fails the run restarts from the true residual
    (new rhat). rho = 0, (rhat, v) = 0 or omega = 0 end the run with BREAKDOWN."""
    b = np.asarray(b, np.float64)
    bb = float(b @ b)
    if bb == 0.0:
        return SolveResult(np.zeros_like(b), 0, OK, 0.0, 0.0)
    thresh = tol * tol * bb
    x = np.zeros_like(b) if x0 is None else np.array(x0, np.float64)
    r = b - A @ x if x0 is not None else b.copy()
    rr = float(r @ r)
    it = 0
    status = NOT_CONVERGED
    restart = True
    while True:
        if restart:
            restart = False
            if rr <= thresh:
                tr = b - A @ x
                trr = float(tr @ tr)
                if trr <= thresh:
                    status = OK
                    break
                r, rr = tr, trr
            rhat = r.copy()
            rho_old = alpha = omega = 1.0
            p = np.zeros_like(b)
            v = np.zeros_like(b)
            rho = float(rhat @ r)
        if it >= max_iter:
            break
        if rho == 0.0:
            status = BREAKDOWN
            break
        beta = (rho / rho_old) * (alpha / omega)
        p = r + beta * (p - omega * v)
        phat = dinv * p
        v = A @ phat
        rv = float(rhat @ v)
        if rv == 0.0:
            status = BREAKDOWN
            break
        alpha = rho / rv
        s = r - alpha * v
        it += 1
        ss = float(s @ s)
        if ss <= thresh:
            x = x + alpha * phat
            r, rr = s, ss
            restart = True
            continue
        shat = dinv * s
        t = A @ shat
        omega = float(t @ s) / float(t @ t)
        x = x + alpha * phat + omega * shat
        r = s - omega * t
        rr = float(r @ r)
        if rr <= thresh:
            restart = True
            continue
        if omega == 0.0:
            status = BREAKDOWN
            break
        rho_old = rho
        rho = float(rhat @ r)
    tr = b - A @ x
    return SolveResult(x, it, status, float(np.sqrt(rr / bb)), float(np.sqrt((tr @ tr) / bb)))


def bicgstab_fp32(A32, dinv32, rhs32, rel_tol=1e-5, max_iter=10000, dtype=np.float32):
    """Inner BiCGStab of the mixed form for the momentum system, x0 = 0.

    The recurrence of ``bicgstab`` (same order of steps, half step when ||s|| is
    small enough) with vectors, values and products in ``dtype``; the dot
    products are accumulated in FP64 and alpha, omega and beta are rounded to
    ``dtype`` before use. No restarts: it stops when the recursive residual
    (||s|| at a half step, else ||r||) is at most rel_tol ||rhs||, on a breakdown
    (rho = 0, (rhat, v) = 0, (t, t) = 0 or omega = 0) or after max_iter
    iterations. Returns (d, iterations, status)."""
    f = dtype

    def dot(u, w):
        return float(u.astype(np.float64) @ w.astype(np.float64))

    d = np.zeros_like(rhs32)
    r = rhs32.copy()
    thresh = rel_tol * rel_tol * dot(r, r)
    if thresh == 0.0 and dot(r, r) == 0.0:
        return d, 0, OK
    rhat = r.copy()
    rho_old = alpha = omega = 1.0
    p = np.zeros_like(r)
    v = np.zeros_like(r)
    rho = dot(rhat, r)
    it = 0
    while it < max_iter:
        if rho == 0.0:
            return d, it, BREAKDOWN
        beta = f((rho / rho_old) * (alpha / omega))
        p = r + beta * (p - f(omega) * v)
        phat = dinv32 * p
        v = A32 @ phat
        rv = dot(rhat, v)
        if rv == 0.0:
            return d, it, BREAKDOWN
        alpha = rho / rv
        s = r - f(alpha) * v
        it += 1
        if dot(s, s) <= thresh:
            return d + f(alpha) * phat, it, OK
        shat = dinv32 * s
        t = A32 @ shat
        tt = dot(t, t)
        if not tt > 0.0:
            return d, it, BREAKDOWN
        omega = dot(t, s) / tt
        d = d + f(alpha) * phat + f(omega) * shat
        r = s - f(omega) * t
        if dot(r, r) <= thresh:
            return d, it, OK
        if omega == 0.0:
            return d, it, BREAKDOWN
        rho_old = rho
        rho = dot(rhat, r)
    return d, it, NOT_CONVERGED


def bicgstab_mixed_ir(A64, A32, dinv32, b, tol=1e-9, inner_tol=1e-5, max_outer=50, max_iter=10000,
                      dtype=np.float32) -> SolveResult:
    """FP32-inner / FP64-outer iterative refinement around BiCGStab.

    x = 0; repeat: r = b - A x with FP64 values; stop when ||r|| <= tol ||b||;
    solve A32 d = fl(r) by ``bicgstab_fp32`` to inner_tol relative (a new
    shadow residual every time); x += d in FP64. ``max_iter`` bounds the inner
    iterations of all passes together."""
    b = np.asarray(b, np.float64)
    bb = float(b @ b)
    x = np.zeros_like(b)
    if bb == 0.0:
        return SolveResult(x, 0, OK, 0.0, 0.0, 0)
    total = 0
    status = NOT_CONVERGED
    outer = 0
    while True:
        r = b - A64 @ x
        rr = float(r @ r)
        if rr <= tol * tol * bb:
            status = OK
            break
        if outer >= max_outer or total >= max_iter:
            break
        d, it, st = bicgstab_fp32(A32, dinv32, r.astype(dtype), inner_tol, max_iter - total, dtype)
        total += it
        outer += 1
        if st == BREAKDOWN:
            status = BREAKDOWN
            break
        x += d.astype(np.float64)
    rel = float(np.sqrt(rr / bb))
    return SolveResult(x, total, status, rel, rel, outer)


def pcg_fp32(A32, dinv32, rhs32, rel_tol=1e-5, max_iter=10000, dtype=np.float32, stop_abs=0.0):
    """Inner PCG of the mixed form, x0 = 0, in working precision ``dtype``.

    The steps of ``pcg`` without restarts: vectors, values and products are
    ``dtype`` (FP32 in the mixed form); the dot products are accumulated in
    FP64 and alpha / beta are rounded to ``dtype`` before use. Stops when the
    recursive residual satisfies ||r|| <= max(rel_tol ||rhs||, stop_abs), on
    a breakdown (p.Ap <= 0) or after max_iter iterations. With dtype FP64 and
    rel_tol = stop_abs = 0 it is ``pcg`` itself, iterate for iterate.
    Returns (d, iterations, status)."""
    prec = _operator(dinv32)
    f = dtype

    def dot(u, w):
        return float(u.astype(np.float64) @ w.astype(np.float64))

    x = np.zeros_like(rhs32)
    r = rhs32.copy()
    rr0 = dot(r, r)
    if rr0 == 0.0:
        return x, 0, OK
    thresh = max(rel_tol * rel_tol * rr0, stop_abs * stop_abs)
    z = prec(r)
    p = z.copy()
    rz = dot(r, z)
    it = 0
    while it < max_iter:
        q = A32 @ p
        pq = dot(p, q)
        if not pq > 0.0:
            return x, it, BREAKDOWN
        alpha = f(rz / pq)
        x += alpha * p
        r -= alpha * q
        it += 1
        if dot(r, r) <= thresh:
            return x, it, OK
        z = prec(r)
        rz_new = dot(r, z)
        beta = f(rz_new / rz)
        p = z + beta * p
        rz = rz_new
    return x, it, NOT_CONVERGED


def mixed_ir(A64, A32, dinv32, b, tol=1e-9, inner_tol=1e-5, max_outer=50, max_inner=10000,
             dtype=np.float32, last_pass=0.5) -> SolveResult:
    """FP32-inner / FP64-outer iterative refinement.

    x = 0; repeat: r = b - A x with FP64 values; stop when ||r|| <= tol ||b||;
    solve A32 d = fl(r) by ``pcg_fp32`` (working precision ``dtype``) from
    d = 0 to ||r_inner|| <= max(inner_tol ||fl(r)||, last_pass tol ||b||);
    x += d in FP64. The second bound keeps the last pass from solving far past
    the outer target: once a reduction by inner_tol would overshoot it, the
    inner solve stops at a fraction ``last_pass`` of the target (0: no cap).
    ``max_inner`` caps each inner solve."""
    b = np.asarray(b, np.float64)
    bb = float(b @ b)
    x = np.zeros_like(b)
    if bb == 0.0:
        return SolveResult(x, 0, OK, 0.0, 0.0, 0)
    stop_abs = last_pass * tol * float(np.sqrt(bb))
    inner_total = 0
    status = NOT_CONVERGED
    outer = 0
    while True:
        r = b - A64 @ x
        rr = float(r @ r)
        if rr <= tol * tol * bb:
            status = OK
            break
        if outer >= max_outer:
            break
        d, it, st = pcg_fp32(A32, dinv32, r.astype(dtype), inner_tol, max_inner, dtype, stop_abs)
        inner_total += it
        outer += 1
        if st == BREAKDOWN:
            status = BREAKDOWN
            break
        x += d.astype(np.float64)
    rel = float(np.sqrt(rr / bb))
    return SolveResult(x, inner_total, status, rel, rel, outer)


def mixed_reliable(A64, A_in, dinv_in, b, tol=1e-9, delta=1e-5, max_iter=20000, max_updates=100,
                   dtype=np.float32) -> SolveResult:
    """Refinement whose inner CG is not restarted ("reliable updates").

    The inner CG runs in ``dtype`` on A_in (values, vectors, products; dot
    products accumulated in FP64, alpha and beta rounded to ``dtype``). When
    its recursive residual has fallen below ``delta`` times the residual at the
    last refinement (or below half the outer target tol ||b||), the inner
    iterate d is added to the FP64 solution
    (x += d, d = 0), the FP64 residual r = b - A64 x is computed and the
    convergence test ||r|| <= tol ||b|| is taken on it; otherwise r replaces
    the inner residual and the iteration CONTINUES with p = z + beta p,
    beta = (r.z)_new / (r.z)_old (no restart of the search direction)."""
    prec = _operator(dinv_in)
    f = dtype
    b = np.asarray(b, np.float64)
    bb = float(b @ b)
    x = np.zeros_like(b)
    if bb == 0.0:
        return SolveResult(x, 0, OK, 0.0, 0.0, 0)
    thresh = tol * tol * bb
    r = b.astype(f)
    r64 = r.astype(np.float64)

    def phase_end(start_rr):
        # the inner tolerance, or half the outer target: a residual just above
        # the target must still make real progress, so it cannot trigger
        # endless one-step phases
        return max(delta * delta * start_rr, 0.25 * thresh)

    inner = phase_end(float(r64 @ r64))
    z = prec(r)
    p = z.copy()
    rz = float(r64 @ z.astype(np.float64))
    d = np.zeros_like(r)
    it = updates = 0
    status = NOT_CONVERGED
    rr = bb
    while True:
        q = A_in @ p
        pq = float(p.astype(np.float64) @ q.astype(np.float64))
        if not pq > 0.0:
            status = BREAKDOWN
            break
        alpha = f(rz / pq)
        d += alpha * p
        r -= alpha * q
        it += 1
        r64 = r.astype(np.float64)
        if float(r64 @ r64) <= inner or it >= max_iter:
            x += d.astype(np.float64)
            d[:] = 0
            res = b - A64 @ x
            rr = float(res @ res)
            updates += 1
            if rr <= thresh:
                status = OK
                break
            if it >= max_iter or updates >= max_updates:
                break
            r = res.astype(f)
            r64 = r.astype(np.float64)
            inner = phase_end(float(r64 @ r64))
        z = prec(r)
        rz_new = float(r64 @ z.astype(np.float64))
        beta = f(rz_new / rz)
        p = z + beta * p
        rz = rz_new
    rel = float(np.sqrt(rr / bb))
    return SolveResult(x, it, status, rel, rel, updates)


# --------------------------------------------------------------------------
# The mixed forms on the symmetrically scaled system
# --------------------------------------------------------------------------
#
# Jacobi preconditioning made explicit: with S = diag(s), s_i = 1/sqrt(a_ii),
# A_hat = S A S has a unit diagonal, and CG on A_hat y = S r with no
# preconditioner is Jacobi-PCG on A d = r with d = S y: the same iterates in
# exact arithmetic (z = D^-1 r becomes r_hat = S r). The inner FP32 solves of
# both refinement forms can run on A_hat; the FP64 residual and update stay
# on A. s is kept in FP64, so the FP32 copy of A_hat has an exactly unit
# diagonal.


def jacobi_scaling(diag):
    """s_i = 1 / sqrt(a_ii) in FP64 (correctly rounded square root and division)."""
    d = np.asarray(diag, np.float64)
    return 1.0 / np.sqrt(d)


def scaled_fp32_values(row_ptr, col_idx, vals, s):
    """FP32 values of S A S: v_ij = fl32(a_ij (s_i s_j)), all products in FP64,
    s_i s_j first (the same rounded product for (i, j) and (j, i), so a
    symmetric A gives an exactly symmetric scaled matrix). The diagonal
    a_ii s_i s_i lies within a few FP64 rounding errors of 1 and is 1 in FP32."""
    n = row_ptr.shape[0] - 1
    row = np.repeat(np.arange(n), np.diff(row_ptr))
    sd = np.asarray(s, np.float64)
    return (np.asarray(vals, np.float64) * (sd[row] * sd[np.asarray(col_idx, np.int64)])).astype(np.float32)


def _scaled_rhs(sd, r, dtype):
    """fl(S r): the FP64 residual scaled in FP64, rounded to the working precision."""
    return (sd * r).astype(dtype)


def mixed_ir_scaled(A64, A_hat, s, b, tol=1e-9, inner_tol=1e-5, max_outer=50, max_inner=10000,
                    dtype=np.float32, last_pass=0.5) -> SolveResult:
    """``mixed_ir`` with its inner solves on the scaled system.

    x = 0; repeat: r = b - A x with FP64 values; stop when ||r|| <= tol ||b||;
    solve A_hat y = fl(S r) by ``pcg_fp32`` with no preconditioner from y = 0 to
    ||r_inner|| <= max(inner_tol ||fl(S r)||, last_pass tol ||b|| c), where
    c = ||fl(S r)|| / ||r|| carries the outer target into the scaled norm;
    x += S y in FP64."""
    b = np.asarray(b, np.float64)
    bb = float(b @ b)
    x = np.zeros_like(b)
    if bb == 0.0:
        return SolveResult(x, 0, OK, 0.0, 0.0, 0)
    sd = np.asarray(s, np.float64)
    inner_total = 0
    status = NOT_CONVERGED
    outer = 0
    while True:
        r = b - A64 @ x
        rr = float(r @ r)
        if rr <= tol * tol * bb:
            status = OK
            break
        if outer >= max_outer:
            break
        rh = _scaled_rhs(sd, r, dtype)
        rh64 = rh.astype(np.float64)
        stop_abs = last_pass * tol * float(np.sqrt(bb)) * float(np.sqrt((rh64 @ rh64) / rr))
        y, it, st = pcg_fp32(A_hat, lambda v: v, rh, inner_tol, max_inner, dtype, stop_abs)
        inner_total += it
        outer += 1
        if st == BREAKDOWN:
            status = BREAKDOWN
            break
        x += sd * y.astype(np.float64)
    rel = float(np.sqrt(rr / bb))
    return SolveResult(x, inner_total, status, rel, rel, outer)


def mixed_reliable_scaled(A64, A_hat, s, b, tol=1e-9, delta=0.1, max_iter=20000, max_updates=100,
                          dtype=np.float32) -> SolveResult:
    """``mixed_reliable`` with its inner CG on the scaled system.

    The inner CG (no preconditioner: z = r_hat) runs in ``dtype`` on A_hat
    from the scaled residual r_hat = fl(S r); dot products accumulated in
    FP64, alpha and beta rounded to ``dtype``. A phase ends when ||r_hat|| has
    fallen by ``delta`` since the phase began, or below half the outer target
    carried into the scaled norm, 0.5 tol ||b|| ||r_hat_0|| / ||r_0|| (r_0,
    r_hat_0: the phase's starting residuals). Then the inner iterate enters the
    solution as x += S y (FP64, y = 0), r = b - A64 x is computed, the
    convergence test ||r|| <= tol ||b|| is taken on it, and otherwise fl(S r)
    replaces the inner residual and the iteration continues with
    p = r_hat + beta p, beta = (r_hat.r_hat)_new / (r_hat.r_hat)_old."""
    f = dtype
    b = np.asarray(b, np.float64)
    bb = float(b @ b)
    x = np.zeros_like(b)
    if bb == 0.0:
        return SolveResult(x, 0, OK, 0.0, 0.0, 0)
    thresh = tol * tol * bb
    sd = np.asarray(s, np.float64)

    def dot(u, w):
        return float(u.astype(np.float64) @ w.astype(np.float64))

    def phase_end(rh, r):
        rh2 = dot(rh, rh)
        return max(delta * delta * rh2, 0.25 * thresh * rh2 / float(r @ r))

    res = b.copy()
    rh = _scaled_rhs(sd, res, f)
    inner = phase_end(rh, res)
    p = rh.copy()
    rz = dot(rh, rh)
    y = np.zeros_like(rh)
    it = updates = 0
    status = NOT_CONVERGED
    rr = bb
    while True:
        q = A_hat @ p
        pq = dot(p, q)
        if not pq > 0.0:
            status = BREAKDOWN
            break
        alpha = f(rz / pq)
        y += alpha * p
        rh -= alpha * q
        it += 1
        rz_new = dot(rh, rh)
        if rz_new <= inner or it >= max_iter:
            x += sd * y.astype(np.float64)
            y[:] = 0
            res = b - A64 @ x
            rr = float(res @ res)
            updates += 1
            if rr <= thresh:
                status = OK
                break
            if it >= max_iter or updates >= max_updates:
                break
            rh = _scaled_rhs(sd, res, f)
            inner = phase_end(rh, res)
            rz_new = dot(rh, rh)
        beta = f(rz_new / rz)
        p = rh + beta * p
        rz = rz_new
    rel = float(np.sqrt(rr / bb))
    return SolveResult(x, it, status, rel, rel, updates)


# --------------------------------------------------------------------------
# Adjoint and gradients
# --------------------------------------------------------------------------


def transpose_values(vals, tpos):
    """Values of A^T in A's pattern: valsT[p] = vals[tpos[p]]."""
    return vals[tpos]


def entry_grad(row_ptr, col_idx, lam, x):
    """dL/da_ij = -lambda_i x_j for every stored entry (from A x = b and
    A^T lambda = dL/dx)."""
    n = row_ptr.shape[0] - 1
    row_of = np.repeat(np.arange(n), np.diff(row_ptr))
    return -lam[row_of] * x[col_idx]


def slot_grad(src_of, g_entry, n_slots):
    """Gradient per buffer slot: the sum over CSR positions fed by the slot."""
    return np.bincount(src_of, weights=g_entry, minlength=n_slots)


def face_grad_ldu(ranks, lam, x):
    """Gradient w.r.t. a face coefficient a_f entering as +a_f on both
    diagonals and -a_f on both off-diagonals: -(lam_l - lam_u)(x_l - x_u).
    Returns per rank [internal faces | interface entries], rank after rank."""
    off = rank_offsets(ranks)
    out = []
    for r, d in enumerate(ranks):
        lo = np.asarray(d.lower_addr, np.int64) + off[r]
        up = np.asarray(d.upper_addr, np.int64) + off[r]
        out.append(-(lam[lo] - lam[up]) * (x[lo] - x[up]))
        i = off[r] + np.asarray(d.iface_row, np.int64)
        j = off[np.asarray(d.iface_nbr_rank, np.int64)] + np.asarray(d.iface_nbr_col, np.int64)
        out.append(-(lam[i] - lam[j]) * (x[i] - x[j]))
    return np.concatenate(out) if out else np.zeros(0)
