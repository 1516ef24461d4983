"""Served batched form vs the plain one-solve-at-a-time path.

``python -m paper_2606_31707_b300.serve_bench [--requests N] [--rate R] [--slots S]``

Requests arrive as a Poisson stream (seeded) with grid sizes drawn from the
D2Q9 grids {200x80, 800x320, 2000x800} and the D3Q19 grids {128^3,
256x128x64}, a seeded porous cylinder each and Re in [20, 200].  Every
request is one mean-flow sensitivity solve with a fixed budget (2000 warm-up
+ 2000 averaging steps, adjoint to 1e-6 or 4000 iterations) in FP32.

* plain: one solve after the other, in arrival order (a request waits for
  the previous one to finish);
* served: the continuous-batching server, requests submitted at their
  arrival times, up to ``slots`` solves running concurrently.

Prints one JSON line with gradients/s and p50/p99 latency of both, and the
largest relative gradient difference between them (the served results are
expected to be identical when both use the same adjoint solver).  With
``--served-solver gmres`` the served form solves the same adjoint fixed point
by restarted GMRES; ``--accuracy`` then also solves every request untimed to a
tighter tolerance and reports each form's largest relative gradient error
against that reference, the accuracy at which the two are compared.
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


def run(args):
    reqs = build_requests(args.requests, args.rate, args.seed, args.warm, args.avg, args.max_iter)
    # warm-up: one small solve to load kernels
    solve_one(build_requests(1, args.rate, 99, 50, 50, 20)[0][1])

    # plain path: sequential in arrival order
    t0 = time.perf_counter()
    plain = []
    lat_plain = []
    clock = 0.0
    per_size = {}
    for t_arr, r in reqs:
        start = max(clock, t_arr)
        t = time.perf_counter()
        res = solve_one(r)
        dt = time.perf_counter() - t
        clock = start + dt
        lat_plain.append(clock - t_arr)
        plain.append(res)
        per_size.setdefault("x".join(map(str, r.dims)), []).append(round(dt, 4))
    wall_plain = time.perf_counter() - t0
    span_plain = clock - reqs[0][0]

    # served path: submit at arrival times, in the chosen storage and solver form
    import dataclasses
    st_code = {"fp32": H.FP32, "fp16dev": H.FP16DEV, "bf16dev": H.BF16DEV}[args.served_storage]
    solver_code = 1 if args.served_solver == "gmres" else 0
    srv = SensitivityServer(slots=args.slots, hbm_budget=args.budget_gb << 30)
    t0 = time.perf_counter()
    futs = []
    for t_arr, r in reqs:
        r = dataclasses.replace(r, storage=st_code, adjoint_solver=solver_code)
        now = time.perf_counter() - t0
        if t_arr > now:
            time.sleep(t_arr - now)
        futs.append(srv.submit(r))
    served = [f.result() for f in futs]
    t_end = time.perf_counter() - t0
    pool = {"hits": srv.pool.hits, "misses": srv.pool.misses} if srv.pool is not None else None
    srv.close()
    lat_served = [s.latency_s for s in served]
    span_served = t_end - reqs[0][0]

    maxdiff = 0.0
    for a, b in zip(plain, served):
        den = float(np.linalg.norm(a.gradient)) or 1.0
        maxdiff = max(maxdiff, float(np.linalg.norm(a.gradient - b.gradient)) / den)
    accuracy = None
    if args.accuracy:
        # untimed reference: the same requests, adjoint by GMRES to a tighter tolerance
        ref = [solve_one(dataclasses.replace(r, adjoint_solver=1, tol=args.ref_tol,
                                             max_iter=args.ref_max_iter)) for _, r in reqs]

        def worst(results):
            e = 0.0
            for a, b in zip(results, ref):
                den = float(np.linalg.norm(b.gradient)) or 1.0
                e = max(e, float(np.linalg.norm(a.gradient - b.gradient)) / den)
            return e
        accuracy = {"reference": {"solver": "gmres", "tol": args.ref_tol,
                                  "max_iter": args.ref_max_iter,
                                  "residuals": [r.adjoint_residual for r in ref]},
                    "plain_max_rel_err": worst(plain), "served_max_rel_err": worst(served)}
    lups = sum(r.lups for r in plain)
    line = {
        "metric": "served gradients/s and p50/p99 latency vs one solve at a time",
        "requests": args.requests, "rate_per_s": args.rate, "slots": args.slots,
        "budget": {"warm_steps": args.warm, "avg_steps": args.avg,
                   "adjoint_max_iter": args.max_iter, "tol": 1e-6, "storage": "fp32"},
        "plain": {"gradients_per_s": len(plain) / span_plain, "p50_s": pct(lat_plain, 50),
                  "p99_s": pct(lat_plain, 99), "busy_s": wall_plain},
        "served": {"gradients_per_s": len(served) / span_served, "p50_s": pct(lat_served, 50),
                   "p99_s": pct(lat_served, 99), "storage": args.served_storage,
                   "adjoint_solver": args.served_solver,
                   "adjoint_iters": [r.adjoint_iters for r in served]},
        "accuracy": accuracy,
        "speedup_gradients_per_s": (len(served) / span_served) / (len(plain) / span_plain),
        "max_rel_gradient_diff_served_vs_plain": maxdiff,
        "mlups_plain": lups / wall_plain / 1e6,
        "plain_solve_s_by_size": per_size,
        "adjoint_iters": [r.adjoint_iters for r in plain],
        "context_pool": pool,
        "sizes": [list(r.dims) for _, r in reqs],
    }
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--requests", type=int, default=16)
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--slots", type=int, default=6)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--warm", type=int, default=2000)
    ap.add_argument("--avg", type=int, default=2000)
    ap.add_argument("--max-iter", type=int, default=4000)
    ap.add_argument("--budget-gb", type=int, default=200)
    ap.add_argument("--served-storage", default="fp32", choices=["fp32", "fp16dev", "bf16dev"])
    ap.add_argument("--served-solver", default="fixed-point", choices=["fixed-point", "gmres"])
    ap.add_argument("--accuracy", action="store_true")
    ap.add_argument("--ref-tol", type=float, default=1e-8)
    ap.add_argument("--ref-max-iter", type=int, default=40000)
    run(ap.parse_args())


if __name__ == "__main__":
    main()
