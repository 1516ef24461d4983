"""Drag of the 2D Schaefer-Turek cylinder (Re = 20) with the cylinder as an
HLBM porous body, d = 0 inside and d = 1 outside (the validation of the
paper's Sec. 5.1; reference c_D = 5.58).

``python -m paper_2606_31707_b300.drag_validation [--N 20 40 80] [--tau 1.0]``

Channel of height H = 4.1 D and length 22 D; the walls are one solid row
(d = 0, with tau = 1 a no-slip node) at y = 0 of the y-periodic domain;
parabolic inflow u(y) = 4 U_m y (H - y) / H^2 through the prescribed-profile
inflow node; cylinder of diameter D = N cells centred (2 D, 2 D) from the
inflow and the lower wall.  The equilibrium inflow node holds rho = 1, so
the flow rate it delivers falls short of the prescribed one by the pressure
drop; the profile is rescaled once so that the mean velocity measured one
diameter downstream of the inflow gives Re = u_mean D / nu = 20.  The force on
the body is the momentum the porous forcing removes per step,
F_x = sum over the body of (1 - d) rho u_x / tau (the force density of the
Brinkman term), and c_D = 2 F_x / (u_mean^2 D).  Prints one JSON line.
Orchestration only: every step runs in the library.
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

from workloads import Regions  # noqa: E402

from . import hlbm as H  # noqa: E402
from .solver import Solver  # noqa: E402

CD_REF = 5.58


def geometry(N: int):
    D = N
    ny = int(round(4.1 * D))
    nx = 22 * D
    xc, yc = 2.0 * D, 2.0 * D
    y, x = np.mgrid[0:ny, 0:nx]
    d = np.ones((1, ny, nx))
    body = (x - xc) ** 2 + (y - yc) ** 2 < (D / 2.0) ** 2
    d[0][body] = 0.0
    d[0, 0, :] = 0.0
    return d, body, nx, ny


def run_case(N: int, tau: float, flow_throughs: float, storage: int):
    d, body, nx, ny = geometry(N)
    nu = (tau - 0.5) / 3.0
    u_mean_target = 20.0 * nu / N
    yy = np.arange(ny, dtype=np.float64)
    shape = 4.0 * yy * (ny - yy) / ny ** 2          # max 1 at mid-channel
    u_max = 1.5 * u_mean_target
    regions = Regions(ffa_x=nx // 2, ffa_y=(0, ny), ffa_z=(0, 1),
                      diss_box=(0, nx, 0, ny, 0, 1), design_box=(0, nx, 0, ny, 0, 1))
    s = Solver(9, (nx, ny, 1), tau, 0.0, storage=storage, u_in=u_mean_target,
               regions=regions, inflow_profile=u_max * shape[None, :])
    s.set_porosity(d)
    steps = int(flow_throughs * nx / u_mean_target)
    steps -= steps % 2
    history = []
    for it in range(2):
        s.run_primal(steps, 0)
        rho = s.field(H.FIELD_RHO)[0]
        u = s.field(H.FIELD_U)[0][0]
        u_mean = float((rho[1:, N] * u[1:, N]).sum() / ny)
        F = float(((1.0 - d[0]) * rho * u)[body].sum() / tau)
        cd = 2.0 * F / (u_mean ** 2 * N)
        history.append(dict(u_mean=u_mean, Re=u_mean * N / nu, F=F, cd=cd))
        if it == 0:
            u_max *= u_mean_target / u_mean
            s.configure(tau, 0.0, u_in=u_mean_target, regions=regions,
                        inflow_profile=u_max * shape[None, :])
    # a second window with the final profile shows the drag is steady
    s.run_primal(steps // 4 - (steps // 4) % 2, 0)
    rho = s.field(H.FIELD_RHO)[0]
    u = s.field(H.FIELD_U)[0][0]
    F2 = float(((1.0 - d[0]) * rho * u)[body].sum() / tau)
    s.close()
    last = history[-1]
    return dict(N=N, grid=[nx, ny], tau=tau, steps_per_window=steps, Ma=u_max / math.sqrt(1 / 3),
                Re=last["Re"], cd=last["cd"], rel_err=abs(last["cd"] - CD_REF) / CD_REF,
                drag_change_last_window=abs(F2 - last["F"]) / abs(last["F"]), history=history)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--N", type=int, nargs="+", default=[20, 40, 80])
    ap.add_argument("--tau", type=float, default=1.0)
    ap.add_argument("--flow-throughs", type=float, default=4.0)
    ap.add_argument("--storage", default="fp32", choices=["fp32", "fp64"])
    args = ap.parse_args()
    st = H.FP32 if args.storage == "fp32" else H.FP64
    cases = [run_case(N, args.tau, args.flow_throughs, st) for N in args.N]
    eoc = []
    for a, b in zip(cases, cases[1:]):
        if a["rel_err"] > 0 and b["rel_err"] > 0:
            eoc.append(math.log(a["rel_err"] / b["rel_err"]) / math.log(b["N"] / a["N"]))
    print(json.dumps({"study": "Schaefer-Turek 2D-1 drag, HLBM porous cylinder (Sec. 5.1)",
                      "cd_reference": CD_REF, "cases": cases, "eoc": eoc}))


if __name__ == "__main__":
    main()
