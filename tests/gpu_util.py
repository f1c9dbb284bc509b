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
