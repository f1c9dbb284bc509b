"""Failure detection without a GPU fault: a device wait that runs out.

spin_limit = 0 makes every mbarrier wait of the sliced SpMV give up at once
(its bulk copies are still in flight; FP64 and mixed PCG, FP64 and mixed
BiCGStab), so each block records the timeout,
waits (bounded) for the copies it issued, and the solve ends with
RP_DEVICE_TIMEOUT instead of a result. The context stays usable: with the
default limit restored, the same handle solves exactly as a fresh handle does
(bitwise), so no stale control state or shared memory outlives the timeout.
96^3 rows give every block several chunks, so the producer warp's wait for a
released stage runs out as well as the consumers' waits for data.
"""
import numpy as np
import pytest
import torch

from paper_2510_08536_gb300 import build, repart, synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    repart.load()
    torch.cuda.set_device(0)


def test_wait_runs_out_and_context_survives():
    mesh = synth.box_mesh(96, 96, 96, 2, 2, 2)
    stg = torch.from_numpy(synth.Assembler(mesh).staging(synth.face_coeffs(mesh, 1.0, 100))).to(DEV)
    mstg = torch.from_numpy(synth.momentum_staging(mesh, 0.5, 100)).to(DEV)
    b = torch.from_numpy(synth.uniform_vector(mesh, 0)).to(DEV)
    n = mesh.n_cells
    h = repart.build_repartition(mesh.ranks, spin_limit=0)
    assert repart.sliced_sizes(h) is not None
    repart.update_values_packed(h, stg)
    for precision in ("fp64", "mixed", "mixed_ru"):
        x = torch.zeros(n, dtype=torch.float64, device=DEV)
        with pytest.raises(repart.RepartError) as e:
            repart.solve(h, b, x, tol=1e-9, precision=precision)
        assert e.value.status == repart.RP_DEVICE_TIMEOUT, precision
    repart.update_values_packed(h, mstg)
    for precision in ("fp64", "mixed"):
        x = torch.zeros(n, dtype=torch.float64, device=DEV)
        with pytest.raises(repart.RepartError) as e:
            repart.solve_bicgstab(h, b, x, tol=1e-9, precision=precision)
        assert e.value.status == repart.RP_DEVICE_TIMEOUT, precision
    torch.cuda.synchronize()

    # the default limit restored: the same handle matches a fresh one bit for bit
    repart.set_solver_options(h, spin_limit=repart.default_options().spin_limit)
    fresh = repart.build_repartition(mesh.ranks)
    for hh in (h, fresh):
        repart.update_values_packed(hh, stg)
    for precision in ("fp64", "mixed_ru"):
        xs = [torch.zeros(n, dtype=torch.float64, device=DEV) for _ in range(2)]
        infos = [repart.solve(hh, b, xx, tol=1e-9, precision=precision) for hh, xx in zip((h, fresh), xs)]
        assert infos[0] == infos[1] and infos[0]["status"] == 0
        assert torch.equal(xs[0], xs[1])
    for hh in (h, fresh):
        repart.update_values_packed(hh, mstg)
    for precision in ("fp64", "mixed"):
        xs = [torch.zeros(n, dtype=torch.float64, device=DEV) for _ in range(2)]
        infos = [repart.solve_bicgstab(hh, b, xx, tol=1e-9, precision=precision) for hh, xx in zip((h, fresh), xs)]
        assert infos[0] == infos[1] and infos[0]["status"] == 0, precision
        assert torch.equal(xs[0], xs[1]), precision
    h.close()
    fresh.close()
