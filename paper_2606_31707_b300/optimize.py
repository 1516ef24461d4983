"""Gradient-based porosity optimisation driven by the adjoint gradient.

The paper computes sensitivities only and names their use in a gradient-based
topology optimisation as future work.  This driver closes that loop on top of
the C ABI: each iteration runs Algorithm 1 (primal with averages, adjoint,
gradient dJ/dd over the design box) and takes a projected steepest-descent
step on the porosity inside the design box, d <- clip(d - s * G / max|G|, 0, 1),
with a backtracking step length s.  A volume constraint keeps the mean
porosity of the design box fixed (the step is projected onto zero mean before
clipping).  Orchestration only; all arithmetic of the method runs in the CUDA
library.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List

import numpy as np

from . import hlbm as H
from .solver import Solver


@dataclass
class OptResult:
    porosity: np.ndarray
    history: List[float] = field(default_factory=list)
    steps: List[float] = field(default_factory=list)


def optimise(solver: Solver, d0: np.ndarray, objective: int, primal_steps: int, avg_window: int = 1,
             iterations: int = 10, step: float = 0.2, mode: int = H.ADJ_EXACT, tol: float = 1e-8,
             max_iter: int = 200000, keep_volume: bool = True) -> OptResult:
    """Minimise J over the porosity of the solver's design box."""
    b = list(solver.opt.design_box)
    sl = (slice(b[4], b[5]), slice(b[2], b[3]), slice(b[0], b[1]))
    d = np.array(d0, dtype=np.float64, copy=True)
    res = OptResult(d)

    def evaluate(dd):
        solver.set_porosity(dd)
        H.hlbm_init_equilibrium(solver.ctx)
        solver.run_primal(primal_steps, avg_window)
        return solver.objective(objective)

    J = evaluate(d)
    res.history.append(J)
    for _ in range(iterations):
        solver.solve_adjoint(objective, mode, tol, max_iter)
        G = solver.gradient()
        gmax = float(np.abs(G).max())
        if gmax == 0.0:
            break
        direction = -G / gmax
        if keep_volume:
            direction = direction - direction.mean()
        s = step
        accepted = False
        while s > 1e-4:
            trial = d.copy()
            trial[sl] = np.clip(d[sl] + s * direction, 0.0, 1.0)
            Jt = evaluate(trial)
            if Jt < J:
                d, J, accepted = trial, Jt, True
                break
            s *= 0.5
        if not accepted:
            evaluate(d)  # restore the state of the current design
            break
        res.history.append(J)
        res.steps.append(s)
    res.porosity = d
    return res
