"""Served form vs the plain one-solve-at-a-time path on a Poisson stream.

``python -m paper_2606_31707_b300.serve_bench [--requests N] [--slots S]``

Requests are drawn (seeded) with grid sizes from the D2Q9 grids {200x80,
800x320, 2000x800} and the D3Q19 grids {128^3, 256x128x64}, a seeded porous
cylinder each and Re in [20, 200].  Every request is one mean-flow
sensitivity solve with a fixed budget (2000 warm-up + 2000 averaging steps,
adjoint to 1e-6 or 4000 iterations) in FP32.

* plain: one solve after the other on its own context (each kernel launch
  covers one request); its service times give the plain capacity C in
  gradients/s;
* served: the continuous-batching server (requests of at most 400 000 cells
  stepped together in cohorts through the batched entry points, the others
  on their own contexts and streams concurrently), requests submitted at
  their arrival times scaled to rates of 0.5, 0.9 and 1.5 C and to the
  nominal 200 requests/s.

Prints one JSON line: gradients/s and p50/p99 latency of the plain path and
of the served form at every rate, and the largest relative gradient
difference between served and plain results (the same FP32 arithmetic in
other kernel instances: rounding only).  With ``--accuracy`` every request is
also solved untimed by GMRES to a tighter tolerance, the reference each
form's gradient error is stated against.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from workloads import Regions, serving_porosity, serving_request_stream  # noqa: E402

from . import hlbm as H  # noqa: E402
from .serve import Request, SensitivityServer, solve_one  # noqa: E402


def build_requests(n, rate, seed, warm, avg, max_iter):
    out = []
    for k, r in enumerate(serving_request_stream(n, rate, seed)):
        dims, q, Re = r["dims"], r["q"], r["Re"]
        nx, ny, nz = dims
        d = serving_porosity(dims, r["seed"])
        D = ny / 4.0
        u0 = 0.05
        tau = u0 * D / Re * 3.0 + 0.5    # nu = u0 D / Re, tau = 3 nu + 1/2
        xc = ny / 2.0
        fx = int(min(nx - 3, xc + 5 * D))
        R = Regions(ffa_x=fx, ffa_y=(0, ny), ffa_z=(0, nz),
                    diss_box=(0, nx, 0, ny, 0, nz), design_box=(0, nx, 0, ny, 0, nz))
        out.append((r["t"], Request(q=q, dims=dims, tau=tau, porosity=d, u_in=u0,
                                    warm_steps=warm, avg_steps=avg,
                                    objective=H.OBJ_DRAG_FFA, tol=1e-6, max_iter=max_iter,
                                    regions=R, tag=k)))
    return out


def pct(v, p):
    return float(np.percentile(np.asarray(v), p)) if v else None


def _served(reqs, rate_scale, args):
    """Submit the requests at their arrival times divided by rate_scale."""
    srv = SensitivityServer(slots=args.slots, hbm_budget=args.budget_gb << 30,
                            batch_cells=args.batch_cells)
    t0 = time.perf_counter()
    futs = []
    for t_arr, r in reqs:
        t_arr = t_arr / rate_scale
        now = time.perf_counter() - t0
        if t_arr > now:
            time.sleep(t_arr - now)
        futs.append((t_arr, srv.submit(r)))
    served = [f.result() for _, f in futs]
    t_end = time.perf_counter() - t0
    cohorts = list(srv.cohorts)
    srv.close()
    span = t_end - reqs[0][0] / rate_scale
    lat = [s.latency_s for s in served]
    return served, {"gradients_per_s": len(served) / span, "p50_s": pct(lat, 50),
                    "p99_s": pct(lat, 99), "span_s": span, "cohorts": cohorts}


def run(args):
    reqs = build_requests(args.requests, args.rate, args.seed, args.warm, args.avg, args.max_iter)
    # warm-up: one small solve and one small cohort to load kernels and graphs
    warm = build_requests(2, args.rate, 99, 64, 64, 20)
    solve_one(warm[0][1])
    _served([(0.0, warm[0][1]), (0.0, warm[1][1])], 1.0, args)

    # plain path: one solve at a time; its service time gives the capacity
    plain, service = [], []
    per_size = {}
    for _, r in reqs:
        t = time.perf_counter()
        plain.append(solve_one(r))
        dt = time.perf_counter() - t
        service.append(dt)
        per_size.setdefault("x".join(map(str, r.dims)), []).append(round(dt, 4))
    capacity = len(reqs) / sum(service)
    # plain latency under the nominal arrival stream: a FIFO queue of the service times
    clock, lat_plain = 0.0, []
    for (t_arr, _), dt in zip(reqs, service):
        clock = max(clock, t_arr) + dt
        lat_plain.append(clock - t_arr)
    nominal_rate = len(reqs) / max(reqs[-1][0], 1e-9)

    rates = {}
    served_nominal = None
    for name, scale_to in (("0.5C", 0.5 * capacity), ("0.9C", 0.9 * capacity),
                           ("1.5C", 1.5 * capacity), ("nominal", nominal_rate)):
        res, stat = _served(reqs, scale_to / nominal_rate, args)
        stat["rate_per_s"] = scale_to
        rates[name] = stat
        if name == "nominal":
            served_nominal = res
    maxdiff = 0.0
    for a, b in zip(plain, served_nominal):
        den = float(np.linalg.norm(a.gradient)) or 1.0
        maxdiff = max(maxdiff, float(np.linalg.norm(a.gradient - b.gradient)) / den)
    accuracy = None
    if args.accuracy:
        import dataclasses
        ref = [solve_one(dataclasses.replace(r, adjoint_solver=1, tol=args.ref_tol,
                                             max_iter=args.ref_max_iter)) for _, r in reqs]

        def errs(results):
            out = []
            for a, b in zip(results, ref):
                den = float(np.linalg.norm(b.gradient)) or 1.0
                out.append(float(np.linalg.norm(a.gradient - b.gradient)) / den)
            return out
        accuracy = {"reference": {"solver": "gmres", "tol": args.ref_tol,
                                  "max_iter": args.ref_max_iter,
                                  "residuals": [r.adjoint_residual for r in ref]},
                    "plain_rel_err": errs(plain), "served_rel_err": errs(served_nominal)}
    lups = sum(r.lups for r in plain)
    line = {
        "metric": "served gradients/s and p50/p99 latency vs one solve at a time",
        "requests": args.requests, "slots": args.slots, "batch_cells": args.batch_cells,
        "budget": {"warm_steps": args.warm, "avg_steps": args.avg,
                   "adjoint_max_iter": args.max_iter, "tol": 1e-6, "storage": "fp32"},
        "plain": {"capacity_gradients_per_s": capacity, "p50_s_at_nominal": pct(lat_plain, 50),
                  "p99_s_at_nominal": pct(lat_plain, 99), "busy_s": sum(service),
                  "mlups": lups / sum(service) / 1e6},
        "served": rates,
        "speedup_at_1.5C": rates["1.5C"]["gradients_per_s"] / capacity,
        "speedup_at_nominal": rates["nominal"]["gradients_per_s"] / capacity,
        "max_rel_gradient_diff_served_vs_plain": maxdiff,
        "accuracy": accuracy,
        "plain_solve_s_by_size": per_size,
        "adjoint_iters": [r.adjoint_iters for r in plain],
        "adjoint_status": [r.status for r in plain],
        "sizes": [list(r.dims) for _, r in reqs],
    }
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--requests", type=int, default=32)
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--slots", type=int, default=6)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--warm", type=int, default=2000)
    ap.add_argument("--avg", type=int, default=2000)
    ap.add_argument("--max-iter", type=int, default=4000)
    ap.add_argument("--budget-gb", type=int, default=200)
    ap.add_argument("--batch-cells", type=int, default=400_000,
                    help="requests of at most this many cells are stepped together in cohorts")
    ap.add_argument("--accuracy", action="store_true")
    ap.add_argument("--ref-tol", type=float, default=1e-8)
    ap.add_argument("--ref-max-iter", type=int, default=40000)
    run(ap.parse_args())


if __name__ == "__main__":
    main()
