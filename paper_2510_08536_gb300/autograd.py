"""Differentiable solve: a torch.autograd.Function over the C ABI.

x = A(c)^-1 b, with c the continuous coefficient buffer of
rp_update_values_packed (rank after rank, [diag | upper | lower | iface]) and
b the right-hand side, both float64 device tensors. The forward is the value
update and the solve (Sec. 3 update procedure, Sec. 4 pressure solve); the
backward is the adjoint: A^T lambda = dL/dx (rp_solve_adjoint, FP64), then
dL/db = lambda and dL/dc = the per-slot sums of -lambda_i x_j over the stored
entries each slot feeds (rp_entry_grad). Every step runs in the library's
kernels; this module only orders the calls.

The handle needs want_transpose (general storage) and n_parts = 1. The
backward re-applies the forward's buffer before the adjoint solve, so the
gradient refers to the forward's matrix even if the handle's values changed
in between.
"""
import torch

from . import repart


class RepartSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, buffer, b, h, tol, precision):
        repart.update_values_packed(h, buffer)
        x = torch.zeros_like(b)
        repart.solve(h, b, x, tol=tol, precision=precision, raise_on_status=True)
        ctx.save_for_backward(buffer, x)
        ctx.h, ctx.tol = h, tol
        return x

    @staticmethod
    def backward(ctx, gx):
        buffer, x = ctx.saved_tensors
        h = ctx.h
        repart.update_values_packed(h, buffer)
        lam = torch.zeros_like(x)
        info = repart.solve_adjoint(h, gx.contiguous(), lam, tol=ctx.tol)
        if info["status"] != repart.RP_OK:
            raise repart.RepartError(info["status"], "rp_solve_adjoint (backward)")
        g_buffer = None
        if ctx.needs_input_grad[0]:
            g_buffer = torch.empty_like(buffer)
            repart.entry_grad(h, lam, x, g_buffer)
        return g_buffer, (lam if ctx.needs_input_grad[1] else None), None, None, None


def solve(h, buffer, b, tol: float = 1e-9, precision: str = "fp64"):
    """x = A(buffer)^-1 b, differentiable with respect to buffer and b."""
    return RepartSolve.apply(buffer, b, h, tol, precision)
