"""torch.autograd through the C ABI: dL/db and dL/dc (coefficient buffer) of
L = 0.5 ||x - x_t||^2 with A(c) x = b, against the oracle's adjoint (dense solve
of A^T lambda = x - x_t, entry gradients summed per slot) to 1e-8, and against
central differences of the forward on a few buffer slots (h = 1e-6, solves to
1e-13) to 1e-4 relative."""
import numpy as np
import pytest
import torch

from oracle import repart_oracle as O
from paper_2510_08536_gb300 import autograd, build, repart, synth

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


@pytest.mark.parametrize("precision", ["fp64", "mixed_ru"])
def test_autograd_matches_adjoint_oracle(precision):
    c = Case((16, 12, 10), (2, 2, 2), sigma=0.5)
    h = repart.build_repartition(c.mesh.ranks, want_transpose=True)
    buf = _t(c.staging).requires_grad_()
    b = _t(c.b).requires_grad_()
    xt = _t(synth.uniform_vector(c.mesh, 1))
    x = autograd.solve(h, buf, b, tol=1e-13, precision=precision)
    loss = 0.5 * ((x - xt) ** 2).sum()
    loss.backward()
    xs = np.linalg.solve(c.A.toarray(), c.b)
    AT = O.csr_matrix(c.map.row_ptr, c.map.col_idx, O.transpose_values(c.vals, c.map.tpos))
    lam = np.linalg.solve(AT.toarray(), xs - xt.cpu().numpy())
    slot = O.slot_grad(c.map.src_of, O.entry_grad(c.map.row_ptr, c.map.col_idx, lam, xs), h.n_slots)
    gb, gc = b.grad.cpu().numpy(), buf.grad.cpu().numpy()
    assert np.linalg.norm(gb - lam) / np.linalg.norm(lam) <= 1e-8
    assert np.abs(gc - slot).max() <= 1e-8 * np.abs(slot).max()
    h.close()


def test_autograd_against_central_differences():
    c = Case((12, 10, 8), (2, 2, 1), sigma=0.5, oracle_map=False)
    h = repart.build_repartition(c.mesh.ranks, want_transpose=True)
    buf0 = _t(c.staging)
    b = _t(c.b)
    xt = _t(synth.uniform_vector(c.mesh, 1))

    def loss(buf):
        x = autograd.solve(h, buf, b, tol=1e-13)
        return 0.5 * float(((x - xt) ** 2).sum())

    buf = buf0.clone().requires_grad_()
    x = autograd.solve(h, buf, b, tol=1e-13)
    (0.5 * ((x - xt) ** 2).sum()).backward()
    g = buf.grad.cpu().numpy()
    hstep = 1e-6
    n = c.mesh.n_cells
    for s in (0, 7, n + 3, int(np.argmax(np.abs(g)))):  # a diagonal slot, a face slot, the largest
        e = torch.zeros_like(buf0)
        e[s] = hstep
        fd = (loss(buf0 + e) - loss(buf0 - e)) / (2 * hstep)
        assert abs(fd - g[s]) <= 1e-4 * max(abs(g[s]), 1e-3 * np.abs(g).max()), (s, fd, g[s])
    h.close()
