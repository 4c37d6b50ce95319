"""Differentiable sparse solve x = A^{-1} b (torch.autograd.Function).

Forward: numeric factorization of A's values and the solve (library
kernels).  Backward reuses the stored L and U: one transpose solve
lam = A^{-T} g gives dL/db = lam, and the library's adjoint scatter gives
dL/dA_ij = -lam_i x_j on A's pattern (no dense gradient is formed).

A Solver holds one set of factors.  When the same Solver factored other
values between this forward and its backward (two differentiable solves
before one backward), the backward refactors the values its forward used
before the transpose solve, so every gradient is taken on its own A."""
from __future__ import annotations

import torch

from . import capi
from .solver import Solver, _nrhs, _stream


class HyluSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vals: torch.Tensor, b: torch.Tensor, solver: Solver):
        vals = vals.detach().contiguous()
        b = b.detach().contiguous()
        solver.factor(vals)
        x = solver.solve(b)
        ctx.solver = solver
        ctx.factor_gen = solver.factor_gen
        ctx.save_for_backward(x, vals)
        return x

    @staticmethod
    def backward(ctx, gx: torch.Tensor):
        x, vals = ctx.saved_tensors
        s = ctx.solver
        if s.factor_gen != ctx.factor_gen:
            # the handle's factors belong to later values: restore this A's
            s.factor(vals)
            ctx.factor_gen = s.factor_gen
        g = gx.contiguous()
        lam = s.solve(g, transpose=True)
        dvals = None
        if ctx.needs_input_grad[0]:
            nrhs = _nrhs(lam, s.n)
            dvals = torch.empty(s.nnz, dtype=torch.float64, device=lam.device)
            capi.hylu_grad_values(s.h, lam.data_ptr(), x.data_ptr(), dvals.data_ptr(), nrhs, s.n,
                                  _stream(None))
        db = lam if ctx.needs_input_grad[1] else None
        return dvals, db, None


def solve(vals: torch.Tensor, b: torch.Tensor, solver: Solver) -> torch.Tensor:
    """x = A(vals)^{-1} b on the pattern analysed by `solver`, differentiable
    in vals and b."""
    return HyluSolve.apply(vals, b, solver)
