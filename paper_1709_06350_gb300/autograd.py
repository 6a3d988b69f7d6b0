"""torch.autograd wrapper of the solve: forward = recon_solve, backward =
recon_adjoint (implicit-function theorem, computed by librecon's kernels).

Only marshalling lives here.  The adjoint uses the potential of the handle's
last solve, so a backward pass must run before the same Solver solves again;
the wrapper checks this and raises instead of returning a wrong gradient.
"""
from __future__ import annotations

import torch

from . import recon


class _Solve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, b, solver, tol, max_cycles):
        phi, stats = solver.solve(b.detach().contiguous(), tol=tol, max_cycles=max_cycles)
        solver._generation = getattr(solver, "_generation", 0) + 1
        ctx.solver = solver
        ctx.generation = solver._generation
        return phi

    @staticmethod
    def backward(ctx, gphi):
        s = ctx.solver
        if getattr(s, "_generation", None) != ctx.generation:
            raise RuntimeError("the Solver solved another density after this forward pass; "
                               "run backward before reusing it (or use one Solver per graph node)")
        return s.adjoint(gphi.contiguous()), None, None, None


def solve(b: torch.Tensor, solver: "recon.Solver", tol: float = 1e-10,
          max_cycles: int = 50) -> torch.Tensor:
    """phi(b) with gradients: d loss / d b = recon_adjoint(d loss / d phi)."""
    return _Solve.apply(b, solver, tol, max_cycles)
