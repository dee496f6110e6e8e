"""The coupled simulation plus objective as a torch.autograd.Function.

forward : J(gamma) through lks_forward (LKS + rigid-body march, Algorithm 1 state loop)
backward: dJ/dgamma through lks_adjoint (reverse sweep) and lks_sensitivity; torch only supplies
          the device tensors and the current stream.

The solver keeps the history of its latest forward only, so a backward must come before the next
forward on the same solver; an out-of-order backward raises instead of differentiating the wrong
march.
"""
from __future__ import annotations

import torch

from .lks import Solver


class LKSObjective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, gamma: torch.Tensor, solver: Solver) -> torch.Tensor:
        g = gamma.detach().to(torch.float64).contiguous()
        J = solver.forward(g)
        ctx.solver = solver
        ctx.forward_id = solver.forward_count
        ctx.gamma_shape = gamma.shape
        ctx.gamma_dtype = gamma.dtype
        return torch.tensor(J, dtype=torch.float64, device=gamma.device)

    @staticmethod
    def backward(ctx, gJ: torch.Tensor):
        solver = ctx.solver
        if solver.forward_count != ctx.forward_id:
            raise RuntimeError("LKSObjective.backward: the solver ran another forward after this one and holds "
                               "only the latest history; run each backward before the next forward")
        solver.adjoint(float(gJ.item()))
        out = torch.empty(solver.P.n_design, dtype=torch.float64, device=gJ.device)
        solver.sensitivity(out)
        return out.view(ctx.gamma_shape).to(ctx.gamma_dtype), None


def objective(gamma: torch.Tensor, solver: Solver) -> torch.Tensor:
    """J(gamma) with a hand-written adjoint as its backward."""
    return LKSObjective.apply(gamma, solver)
