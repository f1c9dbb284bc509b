"""Writes reference_solutions.json: oracle solutions of the benchmark
workloads, sampled, for the error reports of the tests and of bench.py.

For each workload (one coefficient draw, rhs U[-1,1] seed 0, x0 = 0):
  * x_ref   -- the oracle's FP64 Jacobi-PCG at relative residual 1e-9, the
               GPU FP64 path's own recurrence and tolerance;
  * x_exact -- the same PCG run to relative residual 1e-13, standing in for
               the exact solution (its distance to A^-1 b is below
               kappa * 1e-13);
both sampled on 1024 seeded row indices, with their full 2-norms and the
full-vector distance between them. The solves run in the oracle's C / OpenMP
restatement (pinned against the Python oracle in test_oracle_pins.py) on the
map and values of the Python oracle; nothing here touches the CUDA path.

    python tests/golden/make_reference_solutions.py [workload ...]
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import pcg_omp as C  # noqa: E402
from oracle import repart_oracle as O  # noqa: E402
from paper_2510_08536_gb300 import synth  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "reference_solutions.json")
SAMPLES = 1024
SAMPLE_SEED = 20251008
DRAW_SEED = 100


def sample_rows(n: int) -> np.ndarray:
    k = min(SAMPLES, n)
    return np.sort(np.random.default_rng(SAMPLE_SEED).choice(n, k, replace=False))


def one(workload: str) -> dict:
    t0 = time.time()
    w = synth.WORKLOADS[workload]
    mesh = synth.workload_mesh(workload)
    stg = synth.Assembler(mesh).staging(synth.face_coeffs(mesh, w["sigma"], DRAW_SEED))
    b = synth.uniform_vector(mesh, 0)
    (m,) = O.repartition_map(mesh.ranks, 1)
    vals = C.update_values(m.src_of, stg)
    dinv = C.jacobi_inverse(m.diag_pos, vals)
    ref = C.pcg(m.row_ptr, m.col_idx, vals, dinv, b, tol=1e-9, max_iter=50000)
    ex = C.pcg(m.row_ptr, m.col_idx, vals, dinv, b, tol=1e-13, max_iter=50000)
    if ref.status != O.OK or ex.status != O.OK:
        raise RuntimeError(f"{workload}: oracle solve did not converge ({ref.status}, {ex.status})")
    idx = sample_rows(mesh.n_cells)
    return {"draw_seed": DRAW_SEED, "rhs_seed": 0, "n": mesh.n_cells,
            "ref_tol": 1e-9, "ref_iterations": ref.iterations, "ref_true_rel_residual": ref.true_rel_residual,
            "exact_tol": 1e-13, "exact_iterations": ex.iterations, "exact_true_rel_residual": ex.true_rel_residual,
            "norm_ref": float(np.linalg.norm(ref.x)), "norm_exact": float(np.linalg.norm(ex.x)),
            "ref_vs_exact": float(np.linalg.norm(ref.x - ex.x) / np.linalg.norm(ex.x)),
            "idx": idx.tolist(), "x_ref": ref.x[idx].tolist(), "x_exact": ex.x[idx].tolist(),
            "seconds": round(time.time() - t0, 1)}


def main(workloads):
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    data["_source"] = ("oracle Jacobi-PCG (C / OpenMP restatement), FP64, x0 = 0, rhs U[-1,1] seed 0, coefficient "
                       f"draw seed {DRAW_SEED}; x_ref at rel. residual 1e-9, x_exact at 1e-13; {SAMPLES} rows "
                       f"sampled with default_rng({SAMPLE_SEED}); written by make_reference_solutions.py")
    for wl in workloads:
        data[wl] = one(wl)
        with open(OUT, "w") as f:
            json.dump(data, f, indent=0, sort_keys=True)
        d = data[wl]
        print(wl, d["ref_iterations"], d["exact_iterations"], d["ref_vs_exact"], d["seconds"], "s", flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or ["plain_fp64_32", "update_128", "mixed_256"])
