"""``torch.autograd.Function`` mapping a porosity field to an objective.

forward(d) runs the primal with the tracking averages (Algorithm 1, primal
part) and returns J_bar; backward(gJ) solves the (mean-flow) adjoint and
contracts the gradient (Eq. gradients_unsteady), returning gJ * dJ/dd.  All
arithmetic runs in the CUDA library; this module only moves tensors.  The
context keeps the averaged state on the device between forward and backward.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Optional

import torch

from . import hlbm as H
from .solver import Solver


@dataclass
class PrimalSpec:
    steps: int                  # primal steps per forward
    avg_window: int = 1         # 1 = steady
    objective: int = H.OBJ_DRAG_FFA
    mode: int = H.ADJ_EXACT
    tol: float = 1e-8
    max_iter: int = 200000
    warm_start: bool = False    # continue from the last state instead of f^eq(1, u_in)
    allow_unconverged: bool = False  # True: return the last iterate at max_iter instead of raising


class HLBMObjective(torch.autograd.Function):
    """J = HLBMObjective.apply(d, solver, spec); d shaped like the grid (nz, ny, nx)
    or flat.  The solver's design box must be the whole domain."""

    @staticmethod
    def forward(ctx, d: torch.Tensor, solver: Solver, spec: PrimalSpec):
        dd = d.detach().to(torch.float64).contiguous().reshape(-1)
        if dd.is_cuda:
            H.hlbm_set_porosity(solver.ctx, dd)
        else:
            H.hlbm_set_porosity(solver.ctx, dd.numpy())
        if not spec.warm_start:
            H.hlbm_init_equilibrium(solver.ctx)
        H.hlbm_run_primal(solver.ctx, spec.steps, spec.avg_window)
        J = H.hlbm_objective(solver.ctx, spec.objective)
        solver.generation += 1
        ctx.generation = solver.generation
        ctx.solver = solver
        ctx.spec = spec
        ctx.shape = d.shape
        ctx.dtype = d.dtype
        ctx.device = d.device
        return torch.tensor(J, dtype=d.dtype, device=d.device)

    @staticmethod
    def backward(ctx, gJ: torch.Tensor):
        s, spec = ctx.solver, ctx.spec
        if s.generation != ctx.generation:
            # the context's averaged state belongs to a later forward (or was
            # changed through the solver): its adjoint is not this J's gradient
            raise H.HlbmError(H.ESTATE, "the solver ran another primal after this forward; "
                              "call backward before reusing the solver")
        st, it, res = H.hlbm_solve_adjoint(s.ctx, spec.objective, spec.mode, spec.tol, spec.max_iter)
        s.last_adjoint = (st, it, res)
        if st == H.NOT_CONVERGED and not spec.allow_unconverged:
            raise H.HlbmError(H.NOT_CONVERGED, f"adjoint not converged after {it} iterations "
                              f"(residual {res:.3e} > tol {spec.tol:.1e}); raise max_iter or set "
                              "allow_unconverged")
        G = torch.empty(s.design_shape, dtype=torch.float64,
                        device=ctx.device if ctx.device.type == "cuda" else "cpu")
        if G.is_cuda:
            H.hlbm_gradient(s.ctx, G)
        else:
            Gn = G.numpy()
            H.hlbm_gradient(s.ctx, Gn)
        G = G.to(ctx.dtype).reshape(ctx.shape)
        return gJ * G, None, None


def objective(d: torch.Tensor, solver: Solver, spec: PrimalSpec) -> torch.Tensor:
    return HLBMObjective.apply(d, solver, spec)
