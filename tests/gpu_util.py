"""Shared set-up for the GPU parity tests: seeded inputs on both sides."""
import numpy as np

from oracle import repart_oracle as O
from paper_2510_08536_gb300 import synth


class Case:
    """A mesh, its staging buffer for one coefficient draw, rhs, and the oracle system."""

    def __init__(self, dims, parts, sigma=0.5, seed=100, symmetric=False, oracle_map=True):
        self.mesh = synth.box_mesh(*dims, *parts)
        self.symmetric = symmetric
        self.asm = synth.Assembler(self.mesh, symmetric)
        self.a = synth.face_coeffs(self.mesh, sigma, seed)
        self.staging = self.asm.staging(self.a)
        self.b = synth.uniform_vector(self.mesh, 0)
        if oracle_map:
            (self.map,) = O.repartition_map(self.mesh.ranks, 1, symmetric)
            self.vals = O.update_values(self.map.src_of, self.staging)
            self.A = O.csr_matrix(self.map.row_ptr, self.map.col_idx, self.vals)
            self.dinv = O.jacobi_inverse(self.map.row_ptr, self.map.col_idx, self.vals, self.map.diag_pos)

    def true_rel_residual(self, x):
        return float(np.linalg.norm(self.b - self.A @ x) / np.linalg.norm(self.b))


# ------------------------------------------------------------------ sliced layout decoding


def decode(view, n):
    """Yield (rows, L, D, table, ids[L,32], cols[L,32], pos[L,32], t) per slice."""
    desc = view["desc"].cpu().numpy().view(np.uint32).reshape(-1, 2).astype(np.int64)
    tinfo = view["tinfo"].cpu().numpy().view(np.uint32).astype(np.int64)
    tabs = view["tabs"].cpu().numpy().astype(np.int64)
    ibuf = view["ibuf"].cpu().numpy()
    pos = view["pos"].cpu().numpy()
    for s in range(view["n_slices"]):
        (x0, y0), (x1, y1) = desc[s], desc[s + 1]
        L = int(x1 - x0) // 32
        w4, t = int(tinfo[s] >> 31), int(tinfo[s] & 0x7FFFFFFF)
        D = int(tabs[t - 1])
        table = tabs[t:t + D]
        per, bits = (8, 4) if w4 else (4, 8)
        nw = (L + per - 1) // per
        assert y1 - y0 == 32 * nw
        assert bool(w4) == (D <= 16)
        words = ibuf[y0:y1].view(np.uint32).reshape(nw, 32).astype(np.int64)
        k = np.arange(L)
        ids = (words[k // per, :] >> (bits * (k % per))[:, None]) & ((1 << bits) - 1)
        rows = s * 32 + np.arange(32)
        yield rows, L, D, table, ids, rows[None, :] + table[ids], pos[x0:x1].reshape(L, 32), t


def check_layout(view, m, n):
    rp, col = m.row_ptr.astype(np.int64), m.col_idx.astype(np.int64)
    assert view["n_slices"] == (n + 31) // 32
    total = 0
    stored = {}  # table content -> its one place in tabs
    for rows, L, D, table, ids, cols, pos, t in decode(view, n):
        valid = rows < n
        lens = np.where(valid, rp[np.minimum(rows + 1, n)] - rp[np.minimum(rows, n - 1)], 0)
        assert L == lens.max()
        assert (ids < D).all()
        expect_tab = []
        for k in range(L):
            for j in range(32):
                if k < lens[j]:
                    off = col[rp[rows[j]] + k] - rows[j]
                    if off not in expect_tab:
                        expect_tab.append(off)
        assert list(table) == expect_tab
        assert stored.setdefault(tuple(expect_tab), t) == t  # equal tables are stored once
        for k in range(L):
            has = k < lens
            csr = np.where(has, rp[np.minimum(rows, n - 1)] + k, -1)
            np.testing.assert_array_equal(pos[k], csr)
            np.testing.assert_array_equal(cols[k][has], col[csr[has]])
            pad = valid & ~has
            assert (table[ids[k][pad]] == 0).all()  # padding names the diagonal
        total += 32 * L
    assert total == view["n_entries"]
    assert len(set(stored.values())) == len(stored)
