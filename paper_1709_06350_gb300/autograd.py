"""torch.autograd wrappers of the solve and of the reconstruction output.

solve: forward = recon_solve, backward = recon_adjoint (implicit-function
theorem, computed by librecon's kernels).  The adjoint uses the potential of
the handle's last solve, so a backward pass must run before the same Solver
solves again; the wrapper checks this and raises instead of returning a
wrong gradient.

displace: forward = recon_displace_fp64 (psi, delta_r), backward =
recon_displace_adjoint at the saved phi and b.  Composed with solve, a loss
on delta_r gets its gradient with respect to b through both paths (b enters
delta_r directly and through phi).

Only marshalling lives here.
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


class _Displace(torch.autograd.Function):
    @staticmethod
    def forward(ctx, phi, b, solver):
        phi_c, b_c = phi.detach().contiguous(), b.detach().contiguous()
        psi, dl = solver.displace_fp64(phi_c, b_c)
        ctx.solver = solver
        ctx.save_for_backward(phi_c, b_c)
        return psi, dl

    @staticmethod
    def backward(ctx, gpsi, gdl):
        phi, b = ctx.saved_tensors
        gp = None if gpsi is None else gpsi.contiguous()
        gd = None if gdl is None else gdl.contiguous()
        gphi, gb = ctx.solver.displace_adjoint(phi, b, gp, gd)
        return gphi, gb, None


def displace(phi: torch.Tensor, b: torch.Tensor, solver: "recon.Solver"):
    """(psi, delta_r)(phi, b) in FP64 with gradients (recon_displace_adjoint)."""
    return _Displace.apply(phi, b, solver)
