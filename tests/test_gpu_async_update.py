"""RP_MEM_HOST_ASYNC value updates and rp_get_solve_info: the next time step's
coefficients are uploaded on the handle's copy stream while the current solve
runs. The overlap must not change a single result."""
import numpy as np
import pytest
import torch

from gpu_util import Case
from oracle import repart_oracle as O
from paper_2510_08536_gb300 import repart, synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)


def _draws(c, k):
    return [torch.from_numpy(c.asm.staging(synth.face_coeffs(c.mesh, 1.0, 100 + t))).pin_memory() for t in range(k)]


def test_async_update_bit_exact():
    c = Case((24, 20, 16), (2, 2, 1), sigma=1.0)
    h = repart.build_repartition(c.mesh.ranks)
    stg = torch.from_numpy(c.staging).pin_memory()
    repart.update_values_packed(h, stg, asynchronous=True)
    torch.cuda.synchronize()
    v = repart.get_values(h)
    np.testing.assert_array_equal(v["vals"].cpu().numpy(), c.vals)
    np.testing.assert_array_equal(v["vals32"].cpu().numpy(), O.to_fp32(c.vals))
    np.testing.assert_array_equal(v["dinv"].cpu().numpy(), c.dinv)
    h.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed_ru"])
def test_pipelined_steps_equal_sequential_steps(precision):
    """Five time steps with three draws cycled through the two staging buffers:
    step t+1's upload is queued before step t's outcome is read. Every step's x
    (host, pinned) and info equal the sequential run's bit for bit."""
    c = Case((32, 24, 20), (2, 2, 1), sigma=1.0, oracle_map=False)
    stg = _draws(c, 3)
    b = torch.from_numpy(c.b).pin_memory()
    n, steps = c.mesh.n_cells, 5
    h = repart.build_repartition(c.mesh.ranks)
    seq = []
    for t in range(steps):
        x = torch.zeros(n, dtype=torch.float64).pin_memory()
        repart.update_values_packed(h, stg[t % 3])
        info = repart.solve(h, b, x, tol=1e-9, precision=precision)
        seq.append((x.clone(), info))
    xs = [torch.zeros(n, dtype=torch.float64).pin_memory() for _ in range(steps)]
    got = []
    repart.update_values_packed(h, stg[0], asynchronous=True)
    for t in range(steps):
        repart.solve(h, b, xs[t], tol=1e-9, precision=precision, wait=False)
        if t + 1 < steps:
            repart.update_values_packed(h, stg[(t + 1) % 3], asynchronous=True)
        got.append(repart.solve_info(h))
    for t in range(steps):
        assert got[t]["status"] == 0, got[t]
        assert got[t] == seq[t][1], t
        assert torch.equal(xs[t], seq[t][0]), t
    h.close()


def test_solve_info_before_any_solve_is_an_error():
    c = Case((6, 5, 4), (1, 1, 1), oracle_map=False)
    h = repart.build_repartition(c.mesh.ranks)
    with pytest.raises(repart.RepartError) as e:
        repart.solve_info(h)
    assert e.value.status == repart.RP_EINVAL
    h.close()
