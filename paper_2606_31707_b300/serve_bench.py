"""Served form vs the plain one-solve-at-a-time path on a Poisson stream.

``python -m paper_2606_31707_b300.serve_bench [--requests N] [--slots S] [--recipe R]``

Requests are drawn (seeded) with grid sizes from the D2Q9 grids {200x80,
800x320, 2000x800} and the D3Q19 grids {128^3, 256x128x64}, a seeded porous
cylinder each and Re in [20, 200].  Every request is one mean-flow
sensitivity solve in FP32: 2000 warm-up + 2000 averaging steps, then the
adjoint of J_FFA by the recipe:

* ``gmres`` (default): restarted GMRES(30) on the adjoint fixed point, 100
  sweep pairs per operator application, to an update criterion of 3e-5 or
  80 000 sweeps (a calibration of the stream at 1e-4 left 3 of 32 requests
  between 1e-3 and 1.6e-3 of the reference; at 3e-5 the largest of ten was
  2.9e-4);
* ``fixed``: the fixed-point iteration with the stream's nominal budget
  (1e-6 or 4000 sweeps), which leaves errors of 1e-2 to 0.25 and diverges
  for the unsteady requests (their mean-flow linearisation has growing
  modes); its requests of at most 400 000 cells go through the batched lane.

* plain: one solve after the other on its own context (each kernel launch
  covers one request); its service times give the plain capacity C in
  gradients/s;
* served: the continuous-batching server (contexts pooled, each request on
  its own stream and host thread, the small fixed-point requests stepped
  together in cohorts through the batched entry points), requests submitted
  at their arrival times scaled to rates of 0.5, 0.9 and 1.5 C and to the
  nominal 200 requests/s.  A request that reuses a pooled context starts its
  adjoint from the previous request's (the adjoint state stays on the device;
  ``--no-warm-start`` turns this off): the same fixed point and tolerance
  from a nearby start.

Accuracy (on by default): every request is also solved untimed by GMRES to
the FP32 floor of the update criterion (tol 1e-9, at most 80 000 sweeps), the
reference each form's gradient error is stated against; the plain path with
the stream's nominal fixed-point budget is timed and measured too, for
context.

Prints one JSON line: gradients/s and p50/p99 latency of the plain path and
of the served form at every rate, the gradient errors of each form, and the
largest relative difference between served and plain gradients (zero from a
cold start: the same arithmetic in the same kernels; within the tolerance
from a warm one).
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


RECIPES = {
    "gmres": dict(adjoint_solver=1, tol=3e-5, max_iter=80_000, gmres_restart=30, gmres_inner=100),
    "fixed": dict(adjoint_solver=0, tol=1e-6, max_iter=4000),
}
REFERENCE = dict(adjoint_solver=1, tol=1e-9, max_iter=80_000, gmres_restart=30, gmres_inner=100)


def build_requests(n, rate, seed, warm, avg, recipe):
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
                                    objective=H.OBJ_DRAG_FFA, regions=R, tag=k,
                                    **RECIPES[recipe])))
    return out


def pct(v, p):
    return float(np.percentile(np.asarray(v), p)) if v else None


def _served(reqs, rate_scale, args):
    """Submit the requests at their arrival times divided by rate_scale."""
    import dataclasses

    srv = SensitivityServer(slots=args.slots, hbm_budget=args.budget_gb << 30,
                            batch_cells=args.batch_cells)
    t0 = time.perf_counter()
    futs = []
    for t_arr, r in reqs:
        r = dataclasses.replace(r, warm_start=not args.no_warm_start)
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


def _plain_pass(reqs):
    results, service, per_size = [], [], {}
    for _, r in reqs:
        t = time.perf_counter()
        results.append(solve_one(r))
        dt = time.perf_counter() - t
        service.append(dt)
        per_size.setdefault("x".join(map(str, r.dims)), []).append(round(dt, 4))
    return results, service, per_size


def _errors(results, ref):
    out = []
    for a, b in zip(results, ref):
        den = float(np.linalg.norm(b.gradient)) or 1.0
        out.append(float(np.linalg.norm(a.gradient - b.gradient)) / den)
    return out


def _err_stats(e):
    return {"max": max(e), "p50": pct(e, 50), "frac_le_1e-3": sum(v <= 1e-3 for v in e) / len(e)}


def run(args):
    import dataclasses

    reqs = build_requests(args.requests, args.rate, args.seed, args.warm, args.avg, args.recipe)
    # warm-up: one small solve and one small served pair to load kernels and graphs
    warm = build_requests(2, args.rate, 99, 64, 64, args.recipe)
    warm = [(t, dataclasses.replace(r, max_iter=400)) for t, r in warm]
    solve_one(warm[0][1])
    _served([(0.0, warm[0][1]), (0.0, warm[1][1])], 1.0, args)

    # plain path: one solve at a time; its service time gives the capacity
    plain, service, per_size = _plain_pass(reqs)
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
    if not args.no_accuracy:
        ref = [solve_one(dataclasses.replace(r, **REFERENCE)) for _, r in reqs]
        budget = [(t, dataclasses.replace(r, **RECIPES["fixed"])) for t, r in reqs]
        fixed, fixed_service = [], []
        for _, r in budget:
            t = time.perf_counter()
            try:
                fixed.append(solve_one(r))
            except H.HlbmError as e:   # the unsteady requests diverge
                fixed.append(e)
            fixed_service.append(time.perf_counter() - t)
        ok = [(a, b) for a, b in zip(fixed, ref) if not isinstance(a, Exception)]
        fixed_err = _errors([a for a, _ in ok], [b for _, b in ok])
        e_plain, e_served = _errors(plain, ref), _errors(served_nominal, ref)
        accuracy = {
            "reference": dict(REFERENCE, solver="gmres",
                              residuals=[r.adjoint_residual for r in ref],
                              sweeps=[r.adjoint_iters for r in ref]),
            "plain_rel_err": e_plain, "served_rel_err": e_served,
            "plain": _err_stats(e_plain), "served": _err_stats(e_served),
            "fixed_point_at_the_nominal_budget": {
                "budget": RECIPES["fixed"],
                "gradients_per_s": len(budget) / sum(fixed_service),
                "diverged": sum(isinstance(a, Exception) for a in fixed),
                "rel_err_of_the_rest": _err_stats(fixed_err) if fixed_err else None},
        }
    lups = sum(r.lups for r in plain)
    line = {
        "metric": "served gradients/s and p50/p99 latency vs one solve at a time",
        "requests": args.requests, "slots": args.slots, "batch_cells": args.batch_cells,
        "recipe": dict(RECIPES[args.recipe], name=args.recipe, warm_steps=args.warm,
                       avg_steps=args.avg, storage="fp32", objective="drag_ffa"),
        "plain": {"capacity_gradients_per_s": capacity, "p50_s_at_nominal": pct(lat_plain, 50),
                  "p99_s_at_nominal": pct(lat_plain, 99), "busy_s": sum(service),
                  "mlups": lups / sum(service) / 1e6},
        "served": rates,
        "speedup_at_1.5C": rates["1.5C"]["gradients_per_s"] / capacity,
        "speedup_at_nominal": rates["nominal"]["gradients_per_s"] / capacity,
        "warm_start": not args.no_warm_start,
        "max_rel_gradient_diff_served_vs_plain": maxdiff,
        "accuracy": accuracy,
        "plain_solve_s_by_size": per_size,
        "adjoint_iters": [r.adjoint_iters for r in plain],
        "served_adjoint_iters": [r.adjoint_iters for r in served_nominal],
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
    ap.add_argument("--recipe", default="gmres", choices=sorted(RECIPES))
    ap.add_argument("--budget-gb", type=int, default=200)
    ap.add_argument("--batch-cells", type=int, default=400_000,
                    help="fixed-point requests of at most this many cells are stepped together "
                         "in cohorts")
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--no-warm-start", action="store_true")
    run(ap.parse_args())


if __name__ == "__main__":
    main()
