"""Forward-sensitivity growth along an unsteady trajectory (the paper's App. C).

``python -m paper_2606_31707_b300.tangent_study [--steps N] [--window W]``

Runs the Karman case (D2Q9 1100x410, Re 100) from the inflow equilibrium
with the tangent-linear step (``hlbm_run_tangent``), seeding the porosity of
one cell on the cylinder surface (the top of the cylinder, where the flow
passes fastest), and prints one JSON line with, per window of W steps, the
instantaneous J_DISS at the window's start (a primal-only pass of the same
trajectory, to show where the vortex street sets in) and the largest
|dJ_DISS/dd| inside it.  ``--seed-after S`` starts the tangent only after S
primal steps, the paper's second experiment (seeding once the street has
developed).  The exact transient sensitivity grows by orders of magnitude
while the wake becomes unstable and keeps growing afterwards, which is why
the paper turns to the mean-flow adjoint.  Orchestration only.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from workloads import make_workload  # noqa: E402

from . import hlbm as H  # noqa: E402
from .solver import Solver  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=150_000)
    ap.add_argument("--window", type=int, default=5_000)
    ap.add_argument("--seed-after", type=int, default=0)
    ap.add_argument("--storage", default="fp32", choices=["fp32", "fp64"])
    args = ap.parse_args()
    W = args.window
    wl = make_workload("karman2d_re100")
    tau = wl.u0 * wl.L / wl.Re * 3.0 + 0.5       # nu = u0 D / Re, tau = 3 nu + 1/2
    st = H.FP32 if args.storage == "fp32" else H.FP64
    up = wl.u_perturb
    u = np.ascontiguousarray((up[:2] + np.array([wl.u0, 0.0])[:, None, None, None]).reshape(2, -1))

    def fresh():
        s = Solver(9, wl.dims, tau, 0.0, storage=st, u_in=wl.u0, regions=wl.regions)
        s.set_porosity(wl.porosity)
        H.hlbm_init_equilibrium(s.ctx, None, u)
        return s

    # instantaneous J_DISS at the start of every window (primal only)
    s = fresh()
    total = args.seed_after + args.steps
    j_hist = []
    for _ in range(0, total, W):
        s.run_primal(1, 1)
        j_hist.append(s.objective(H.OBJ_DISSIPATION))
        s.run_primal(W - 1, 0)
    s.close()
    # one cell on the top of the cylinder surface (d crosses 1/2 there)
    xc, yc, R = 125, 205, 25
    delta = np.zeros(wl.porosity.shape)
    delta[0, yc + R, xc] = 1.0
    s = fresh()
    if args.seed_after:
        s.run_primal(args.seed_after, 0)
    jd = H.hlbm_run_tangent(s.ctx, args.steps, np.ascontiguousarray(delta.ravel()), H.OBJ_DISSIPATION)
    s.close()
    peaks = [float(np.abs(jd[k:k + W]).max()) for k in range(0, len(jd), W)]
    line = {"study": "forward sensitivity growth, Karman case, d(J_DISS)/dd of one surface cell",
            "steps": args.steps, "window": W, "seed_after": args.seed_after,
            "storage": args.storage, "seed_cell_xy": [xc, yc + R],
            "seed_cell_porosity": float(wl.porosity[0, yc + R, xc]),
            "J_diss_at_window_start": j_hist,
            "max_abs_jdot_per_window": peaks,
            "max_over_min_window_peak": max(peaks) / max(min(peaks), 1e-300)}
    print(json.dumps(line))


if __name__ == "__main__":
    main()
