"""Writes iteration_counts.json: the oracle's Jacobi-PCG iteration counts
(FP64, relative residual 1e-9, x0 = 0) for the coefficient draws of the
256^3 / k=128 workload, lognormal(0, 1) faces, rhs U[-1,1] seed 0.

Calls only the CPU oracle and the seeded input generator. The CPU-baseline
leg of bench.py times a bounded number of oracle iterations and scales the
per-iteration time by these counts to a per-time-step figure.

    python tests/golden/make_iteration_counts.py 100 101 102 103
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import repart_oracle as O  # noqa: E402
from paper_2510_08536_gb300 import synth  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "iteration_counts.json")


def main(seeds):
    mesh = synth.workload_mesh("mixed_256")
    asm = synth.Assembler(mesh)
    (m,) = O.repartition_map(mesh.ranks, 1)
    b = synth.uniform_vector(mesh, 0)
    data = json.load(open(OUT)) if os.path.exists(OUT) else {
        "_source": "oracle Jacobi-PCG, FP64, tol 1e-9, x0 = 0; workload mixed_256 (256^3, k=128, lognormal sigma=1.0, rhs seed 0); written by make_iteration_counts.py",
        "mixed_256": {}}
    for seed in seeds:
        t = time.time()
        vals = O.update_values(m.src_of, asm.staging(synth.face_coeffs(mesh, 1.0, seed)))
        A = O.csr_matrix(m.row_ptr, m.col_idx, vals)
        res = O.pcg(A, O.jacobi_inverse(m.row_ptr, m.col_idx, vals, m.diag_pos), b, tol=1e-9)
        data = json.load(open(OUT)) if os.path.exists(OUT) else data
        data["mixed_256"][str(seed)] = {"iterations": res.iterations, "status": res.status,
                                        "true_rel_residual": res.true_rel_residual}
        with open(OUT, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        print(seed, res.iterations, res.status, res.true_rel_residual, f"{time.time() - t:.0f}s", flush=True)


if __name__ == "__main__":
    main([int(s) for s in sys.argv[1:]] or [100])
