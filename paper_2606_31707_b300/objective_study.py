"""Steady adjoint gradients of the three objectives on the Re-20 cylinder,
compared with finite-difference quotients at points on the cylinder surface
(the comparison of the paper's Sec. 5.2: J_MEA, J_FFA, J_DISS).

``python -m paper_2606_31707_b300.objective_study [--steps N] [--h H]``

The D2Q9 200x80 FP64 case is run to a steady state with all three objectives
averaged (window of one step), the adjoint is solved for each, and for each of
eight surface cells (d closest to 1/2 along rays at 0, 45, ..., 315 degrees)
the primal is rerun with d -/+ h at that cell to form the central quotient.
Besides the agreement per objective, the line reports how concentrated the
adjoint field is at the wall: the largest |mu| within two cells of the
surface over the largest |mu| elsewhere.  Orchestration only.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from workloads import make_workload  # noqa: E402

from . import hlbm as H  # noqa: E402
from .solver import Solver  # noqa: E402

OBJS = (("drag_mea", H.OBJ_DRAG_MEA), ("drag_ffa", H.OBJ_DRAG_FFA),
        ("dissipation", H.OBJ_DISSIPATION))


def surface_samples(d, xc, yc, R):
    """Eight cells on the surface: along each ray the cell whose d is closest to 1/2."""
    out = []
    for k in range(8):
        a = 2 * math.pi * k / 8
        best = None
        for r10 in range(int((R - 4) * 10), int((R + 4) * 10)):
            r = r10 / 10
            x, y = int(round(xc + r * math.cos(a))), int(round(yc + r * math.sin(a)))
            v = abs(d[0, y, x] - 0.5)
            if best is None or v < best[0]:
                best = (v, x, y)
        out.append((best[1], best[2]))
    return out


def run_js(wl, tau, d, steps):
    s = Solver(9, wl.dims, tau, 0.0, storage=H.FP64, u_in=wl.u0, regions=wl.regions,
               objectives=H.OBJ_DRAG_FFA | H.OBJ_DISSIPATION | H.OBJ_DRAG_MEA)
    s.set_porosity(d)
    s.run_primal(steps, 1)
    return s, {name: s.objective(o) for name, o in OBJS}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=20_000)
    ap.add_argument("--h", type=float, default=1e-4)
    ap.add_argument("--tol", type=float, default=1e-12)
    args = ap.parse_args()
    wl = make_workload("cyl2d_re20")
    tau = wl.u0 * wl.L / wl.Re * 3.0 + 0.5
    d = wl.porosity
    xc, yc, R = 50.0, 40.0, 10.0
    pts = surface_samples(d, xc, yc, R)
    s, J = run_js(wl, tau, d, args.steps)
    grads, near_far, iters = {}, {}, {}
    nz, ny, nx = d.shape
    yy, xx = np.mgrid[0:ny, 0:nx]
    rr = np.hypot(xx - xc, yy - yc)
    band = np.abs(rr - R) <= 2.0
    for name, o in OBJS:
        st, it, res = s.solve_adjoint(o, H.ADJ_EXACT, args.tol, 2_000_000)
        iters[name] = [int(st), int(it), float(res)]
        G = s.gradient()
        grads[name] = [float(G[0, y, x]) for x, y in pts]
        mu = np.abs(s.field(H.FIELD_LAMBDA)).max(axis=0)[0]
        near_far[name] = float(mu[band].max() / max(mu[~band].max(), 1e-300))
    s.close()
    fd = {name: [] for name, _ in OBJS}
    for x, y in pts:
        jp, jm = [], []
        for sgn, store in ((1, jp), (-1, jm)):
            dd = d.copy()
            dd[0, y, x] += sgn * args.h
            sp, Jv = run_js(wl, tau, dd, args.steps)
            sp.close()
            store.append(Jv)
        for name, _ in OBJS:
            fd[name].append((jp[0][name] - jm[0][name]) / (2 * args.h))
    agree = {}
    for name, _ in OBJS:
        g, f = np.array(grads[name]), np.array(fd[name])
        agree[name] = float(np.abs(g - f).max() / max(np.abs(f).max(), 1e-300))
    line = {"study": "steady adjoint vs central quotients on the cylinder surface (Re 20, D2Q9 200x80, FP64)",
            "steps": args.steps, "h": args.h, "samples_xy": pts,
            "J": J, "adjoint_status_iters_residual": iters,
            "gradient_at_samples": grads, "fd_at_samples": fd,
            "max_rel_dev_adjoint_vs_fd": agree,
            "wall_concentration_max_mu_band_over_rest": near_far}
    print(json.dumps(line))


if __name__ == "__main__":
    main()
