"""Benchmark of the HLBM mean-flow adjoint hot path on B300.

One step = the whole hot path over one synthetic case (default: the D2Q9
unsteady Karman case, 1100x410, Re 100, FP32 populations): porosity upload,
primal warm-up, primal averaging window with the tracking averages of f,
J, dJ/df and dJ/dd, then for the drag (J_FFA) and the dissipation (J_DISS)
objectives: linearisation, mean-flow adjoint to tolerance and gradient.

Prints one JSON line (see the contract in the repository documentation):
value = whole-job lattice updates per second (primal steps + adjoint
iterations, x cells) in MLUPS, measured with CUDA events on the device with
inputs resident; e2e = the same metric through the C ABI with host buffers
and the host<->device copies inside the timed region; roofline of the
dominant kernel against the measured HBM copy bandwidth; cpu_baseline = the
FP64 oracle on a bounded sample of the same workload.

``--impl reference`` times the oracle itself (the only reference there is),
on the host cores, on the same workload and metric.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

# the CPU oracle (cpu_baseline and the reference arm) runs on one host thread:
# numpy elementwise work is single-threaded and BLAS is pinned to one thread here
for _k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_k, "1")

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from workloads import make_workload  # noqa: E402

L2_BYTES = 126 * 2 ** 20
CS2 = 1.0 / 3.0

# DRAM bytes (read + write) per launch measured by ncu for the dominant kernels,
# keyed by a hash of the kernel sources at capture time; a kernel changed since
# its capture reports traffic null.  Summaries: profiles/*.md.
MEASURED_DRAM = {
    # ncu dram__bytes_read.sum + dram__bytes_write.sum, mean of the two AA parities
    # (profiles/k_primal_karman2d_re100.md, k_adjoint_karman2d_re100.md,
    # k_primal_rr_les3d_re3900.md)
    ("31489d5ea0988b20", "karman2d_re100", "fp32", "bgk", "primal_step_accumulate"): 34_510_000,
    ("31489d5ea0988b20", "karman2d_re100", "fp32", "bgk", "primal_step_plain"): 18_050_000,
    ("31489d5ea0988b20", "karman2d_re100", "fp32", "bgk", "adjoint_step_ffa"): 30_270_000,
    ("31489d5ea0988b20", "les3d_re3900", "fp32", "rr", "primal_step_accumulate"): 6_872_420_000,
    ("31489d5ea0988b20", "les3d_re3900", "fp32", "rr", "primal_step_plain"): 3_138_120_000,
}


def kernel_source_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2606_31707_b300", "csrc")
    for name in sorted(os.listdir(csrc)):
        # the translation units that define the hot-path kernels and their headers
        if name in ("hlbm_primal.cu", "hlbm_adjoint.cu", "hlbm_device.cuh", "hlbm_internal.h"):
            with open(os.path.join(csrc, name), "rb") as fh:
                h.update(name.encode() + b"\0" + fh.read())
    return h.hexdigest()[:16]


def tau_of(wl):
    # nu = u0 L / Re, tau = nu / c_s^2 + 1/2 (viscosity-relaxation relation)
    return (wl.u0 * wl.L / wl.Re) / CS2 + 0.5


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="karman2d_re100")
    ap.add_argument("--primal-steps", type=int, default=None,
                    help="override the workload's primal step count (testing only)")
    ap.add_argument("--avg-window", type=int, default=None)
    ap.add_argument("--adjoint-tol", type=float, default=1e-6)
    ap.add_argument("--adjoint-mode", default="exact", choices=["exact", "fta"])
    ap.add_argument("--adjoint-solver", default="fixed-point", choices=["fixed-point", "gmres"],
                    help="the paper's iteration, or restarted GMRES on the same fixed point")
    ap.add_argument("--tau-adj", type=float, default=0.0,
                    help="adjoint relaxation time (0: tau0), the regularisation of Sec. 5.4")
    ap.add_argument("--adjoint-max-iter", type=int, default=20000)
    ap.add_argument("--collision", default=None, choices=["bgk", "rr"],
                    help="BGK (Sec. 2.1) or the recursive regularised collision (Sec. 2.2); "
                         "default: the workload's (rr for the LES cases, else bgk)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--storage", default=None, choices=["fp64", "fp32", "fp16dev", "bf16dev"],
                    help="population storage (default: the workload's)")
    return ap.parse_args()


def storage_code(H, wl):
    return {"fp64": H.FP64, "fp32": H.FP32, "fp16dev": H.FP16DEV, "bf16dev": H.BF16DEV}[wl.storage]


def job_shape(wl, args):
    steps = args.primal_steps or wl.steps
    W = args.avg_window if args.avg_window is not None else min(wl.avg_window, steps)
    return steps, W


# ---------------------------------------------------------------------------
# algorithmic bytes per lattice update
# ---------------------------------------------------------------------------

def bytes_model(wl, storage_bytes, real_bytes, exact_rec=False, rr=False):
    """Algorithmic bytes per lattice update of each kernel (reads + writes).

    Averaging step: the populations and porosity of a plain step plus, for
    each running sum it updates, a read-modify-write of the sum -- 16 B for
    FP64 storage; for the other storages the sample goes to a float staging
    value (8 B) that is folded into the FP64 sum every 64 samples
    (16 B + 8 B, amortised 1.5 B).  Sums: density and momentum (1 + D), all q
    populations and tau_eff - tau0 when Cs > 0, and inside the objective
    regions the dJ/df coefficients (2 on the drag plane, 1 + D + D(D+1)/2 in
    the dissipation box) and dJ/dd.  The regularised collision (rr) keeps the
    D(D+1)/2 second moments instead of the q populations, and its adjoint
    record is rho, u, omega and the stress (2 + D + D(D+1)/2 planes)."""
    q = wl.q
    nx, ny, nz = wl.dims
    N = nx * ny * nz
    D = 2 if q == 9 else 3
    plain = 2 * q * storage_bytes + real_bytes
    r = wl.regions
    ffa_cells = (r.ffa_y[1] - r.ffa_y[0]) * (r.ffa_z[1] - r.ffa_z[0])
    b = r.diss_box
    diss_cells = (b[1] - b[0]) * (b[3] - b[2]) * (b[5] - b[4])
    les = wl.Cs > 0
    sb = 16.0 if real_bytes == 8 else 8.0 + 24.0 / 64
    if rr:
        acc = plain + sb * (1 + D + D * (D + 1) // 2) + (sb if les else 0)
    else:
        acc = plain + sb * (1 + D) + (sb * (q + 1) if les else 0)
    acc += (ffa_cells * sb * 2 + diss_cells * sb * (1 + D + D * (D + 1) // 2 + 1)) / N
    rec = D + 2 + D * (D + 1) // 2 if rr else (q if exact_rec else D + 2)
    adj_ffa = (2 * q + rec + 1) * real_bytes + ffa_cells * q * real_bytes / N
    adj_diss = (2 * q + rec + 1) * real_bytes + diss_cells * q * real_bytes / N
    return dict(plain=plain, acc=acc, adj_ffa=adj_ffa, adj_diss=adj_diss)


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), parts[4:8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for _, _, flags in rows for k, v in enumerate(flags)
                          if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows),
                "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows)}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def max_over_ranks(x: float, world: int, device=None) -> float:
    """Largest value of x over all ranks (the slowest rank's time)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_mlups(lups_per_rank: int, ms_max: float, world: int) -> float:
    """Whole-job throughput: every rank processes its own replica (weak scaling)."""
    return world * lups_per_rank / (ms_max * 1e-3) / 1e6


def run_ours(args, rank, world):
    import torch

    from paper_2606_31707_b300 import Solver
    from paper_2606_31707_b300 import hlbm as H

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    wl = make_workload(args.workload, seed=rank)
    if args.collision is None:
        args.collision = wl.collision
    if args.storage:
        import dataclasses
        wl = dataclasses.replace(wl, storage=args.storage)
    steps, W = job_shape(wl, args)
    n_warm = steps - W
    stream = torch.cuda.Stream(device=dev)
    s = Solver(wl.q, wl.dims, tau_of(wl), wl.Cs, storage=storage_code(H, wl), u_in=wl.u0,
               regions=wl.regions, stream=stream, tau_adj=args.tau_adj,
               adjoint_solver=1 if args.adjoint_solver == "gmres" else 0,
               collision=H.COLL_RR if args.collision == "rr" else H.COLL_BGK)
    mode = H.ADJ_EXACT if args.adjoint_mode == "exact" else H.ADJ_FTA
    N = wl.cells
    D = 2 if wl.q == 9 else 3
    d_dev = torch.from_numpy(np.ascontiguousarray(wl.porosity.ravel())).to(dev)
    up = wl.u_perturb if wl.u_perturb is not None else np.zeros((3,) + wl.porosity.shape)
    u0 = up.copy()
    u0[0] += wl.u0
    u_host = np.ascontiguousarray(u0[:D].reshape(D, -1))
    u_dev = torch.from_numpy(u_host).to(dev)
    b = wl.regions.design_box
    gvol = (b[1] - b[0]) * (b[3] - b[2]) * (b[5] - b[4])
    g_dev = torch.empty((2, gvol), dtype=torch.float64, device=dev)
    g_host = np.empty((2, gvol))
    flush = torch.empty(int(2 * L2_BYTES // 4), dtype=torch.float32, device=dev)
    objectives = (H.OBJ_DRAG_FFA, H.OBJ_DISSIPATION)

    phase = dict(plain_ms=0.0, plain_launch=0, acc_ms=0.0, acc_launch=0, adj_ms=[0.0, 0.0],
                 adj_launch=[0, 0], adj_iters=[0, 0])

    def one_step(host: bool, record: bool):
        if host:
            s.set_porosity(wl.porosity.ravel())
            H.hlbm_init_equilibrium(s.ctx, None, u_host)
        else:
            s.set_porosity(d_dev)
            H.hlbm_init_equilibrium(s.ctx, None, u_dev)
        lups = 0
        if n_warm > 0:
            s.run_primal(n_warm, 0)
            st = s.stats()
            if record:
                phase["plain_ms"] += st.primal_ms
                phase["plain_launch"] += st.primal_launches
        s.run_primal(W, W)
        st = s.stats()
        if record:
            phase["acc_ms"] += st.primal_ms
            phase["acc_launch"] += st.primal_launches
        lups += steps * N
        Js = []
        for k, o in enumerate(objectives):
            Js.append(s.objective(o))
            _, it, res = s.solve_adjoint(o, mode, args.adjoint_tol, args.adjoint_max_iter)
            st = s.stats()
            if record:
                phase["adj_ms"][k] += st.adjoint_ms
                phase["adj_launch"][k] += st.adjoint_launches
                phase["adj_iters"][k] += it
            lups += it * N
            if host:
                H.hlbm_gradient(s.ctx, g_host[k])
            else:
                H.hlbm_gradient(s.ctx, g_dev[k])
        return lups, Js

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    def timed(host: bool):
        for _ in range(args.warmup):
            one_step(host, False)
        phase.update(plain_ms=0.0, plain_launch=0, acc_ms=0.0, acc_launch=0,
                     adj_ms=[0.0, 0.0], adj_launch=[0, 0], adj_iters=[0, 0])
        k0 = s.stats().kernels_total
        total_lups = 0
        ms = 0.0
        barrier()
        for _ in range(args.steps):
            flush.zero_()                       # L2 flush between timed steps
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            t0 = time.perf_counter()
            e0.record(stream)
            lups, Js = one_step(host, True)
            e1.record(stream)
            e1.synchronize()
            wall = (time.perf_counter() - t0) * 1e3
            gpu = e0.elapsed_time(e1)
            ms += wall if host else gpu
            total_lups += lups
        barrier()
        launches = s.stats().kernels_total - k0
        return total_lups, ms, launches, Js

    sampler = ClockSampler(dev.index or 0)
    sampler.start()
    lups, ms, launches, Js = timed(False)
    clocks = sampler.stop()
    phase_dev = {k: (list(v) if isinstance(v, list) else v) for k, v in phase.items()}
    ms = max_over_ranks(ms, world, dev)
    value = job_mlups(lups, ms, world)
    e2e = None
    if not args.no_e2e:
        lups_h, ms_h, _, _ = timed(True)
        ms_h = max_over_ranks(ms_h, world, dev)
        e2e = {"value": job_mlups(lups_h, ms_h, world), "unit": "MLUPS",
               "h2d_bytes_per_step": int(N * 8 + D * N * 8),
               "d2h_bytes_per_step": int(2 * gvol * 8 + 2 * 8)}
    s.close()
    return dict(wl=wl, steps=steps, W=W, value=value, ms=ms, lups=lups, e2e=e2e,
                launches=launches, phase=phase_dev, clocks=clocks, Js=Js)


def roofline_of(res, args, H_storage_bytes, real_bytes):
    wl = res["wl"]
    N = wl.cells
    bm = bytes_model(wl, H_storage_bytes, real_bytes,
                     exact_rec=(wl.Cs > 0 and args.adjoint_mode == "exact"),
                     rr=args.collision == "rr")
    ph = res["phase"]
    cand = []
    if ph["plain_launch"]:
        cand.append(("primal_step_plain", ph["plain_ms"], ph["plain_launch"], bm["plain"]))
    if ph["acc_launch"]:
        cand.append(("primal_step_accumulate", ph["acc_ms"], ph["acc_launch"], bm["acc"]))
    for k, key in enumerate(("adj_ffa", "adj_diss")):
        if ph["adj_launch"][k]:
            cand.append((f"adjoint_step_{key[4:]}", ph["adj_ms"][k], ph["adj_launch"][k], bm[key]))
    name, ms, launches, bpl = max(cand, key=lambda c: c[1])
    per_launch_s = ms * 1e-3 / launches
    achieved = bpl * N / per_launch_s / 1e9
    src_hash = kernel_source_hash()
    traffic = MEASURED_DRAM.get((src_hash, wl.name, wl.storage, args.collision, name))
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    peak = peaks.get("hbm_gbs", 6400.0)
    share = {c[0]: c[1] for c in cand}
    tot = sum(share.values())
    return {"kernel": name, "bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
            "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": traffic,
            "traffic_unit": "bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)",
            "algorithmic_bytes_per_launch": round(bpl * N), "kernel_source_hash": src_hash,
            "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
            "bytes_per_lup": round(bpl, 2), "launch_us": round(per_launch_s * 1e6, 3),
            "time_share": {k: round(v / tot, 4) for k, v in share.items()},
            "phase_mlups": {c[0]: round(N * c[2] / (c[1] * 1e-3) / 1e6, 1) for c in cand}}


# ---------------------------------------------------------------------------
# the oracle on a bounded sample (cpu_baseline and --impl reference)
# ---------------------------------------------------------------------------

def oracle_sample(wl, steps, W, adj_iters, n_plain=10, n_acc=2, n_adj=20, collision="bgk"):
    """Time the oracle on a bounded sample of the workload and extrapolate the
    whole job's LUP mix; returns (MLUPS, seconds spent, description)."""
    import contextlib

    try:
        from threadpoolctl import threadpool_limits
    except ImportError:  # BLAS is already pinned to one thread by the environment
        def threadpool_limits(_n):
            return contextlib.nullcontext()

    from oracle import adjoint as oadj
    from oracle import hlbm as ohlbm
    from oracle import meanflow as omf

    t_start = time.perf_counter()
    with threadpool_limits(1):
        P = ohlbm.Params(wl.q, wl.dims, tau0=ohlbm.tau_from_reynolds(wl.u0, wl.L, wl.Re),
                         Cs=wl.Cs, u_in=wl.u0, collision=collision)
        f = ohlbm.initial_state(P, wl.u_perturb)
        d = wl.porosity
        t = time.perf_counter()
        for _ in range(n_plain):
            f = ohlbm.step(f, d, P)
        t_plain = (time.perf_counter() - t) / n_plain
        t = time.perf_counter()
        out = omf.run_primal(f, d, P, n_acc, n_acc, wl.regions, 3)
        t_acc = (time.perf_counter() - t) / n_acc
        t = time.perf_counter()
        lin = oadj.Linearisation(out["fbar"], d, P, oadj.EXACT, None, out["tau_t_bar"])
        t_lin = time.perf_counter() - t
        g = out[("gbar", 2)]
        t = time.perf_counter()
        oadj.solve_adjoint(lin, g, tol=0.0, max_iter=n_adj)
        t_adj = (time.perf_counter() - t) / n_adj
    spent = time.perf_counter() - t_start
    N = wl.cells
    job_s = (steps - W) * t_plain + W * t_acc + 2 * t_lin + sum(adj_iters) * t_adj
    lups = N * (steps + sum(adj_iters))
    desc = (f"full {wl.dims[0]}x{wl.dims[1]}x{wl.dims[2]} grid: {n_plain} plain steps "
            f"({t_plain:.3f} s each), {n_acc} averaging steps ({t_acc:.3f} s), one "
            f"linearisation ({t_lin:.2f} s), {n_adj} adjoint iterations ({t_adj:.3f} s); "
            f"extrapolated to {steps} primal steps ({W} averaging) + {sum(adj_iters)} adjoint "
            f"iterations + 2 linearisations")
    return lups / job_s / 1e6, spent, desc


def run_reference(args):
    wl = make_workload(args.workload)
    steps, W = job_shape(wl, args)
    adj = [args.adjoint_max_iter, args.adjoint_max_iter]
    vals = []
    for k in range(args.warmup + args.steps):
        v, spent, desc = oracle_sample(wl, steps, W, adj, n_plain=4, n_acc=1, n_adj=8,
                                       collision=args.collision or wl.collision)
        if k >= args.warmup:
            vals.append((v, spent))
    value = statistics.median(v for v, _ in vals)
    ms = statistics.median(sp for _, sp in vals) * 1e3
    line = {"impl": "reference", "metric": "primal/adjoint MLUPS (whole job)", "value": value,
            "unit": "MLUPS", "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.name, "grid": list(wl.dims), "lattice": f"D{2 if wl.q == 9 else 3}Q{wl.q}",
                       "collision": args.collision or wl.collision,
                       "primal_steps": steps, "avg_window": W,
                       "adjoint_iters_assumed": adj},
            "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": 1, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    args = parse()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    if args.impl == "reference":
        if rank == 0:
            run_reference(args)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        dist.init_process_group("nccl")
    res = run_ours(args, rank, world)
    if rank != 0:
        return
    wl = res["wl"]
    sb = {"fp64": 8, "fp32": 4, "fp16dev": 2, "bf16dev": 2}[wl.storage]
    rb = 8 if wl.storage == "fp64" else 4
    roof = roofline_of(res, args, sb, rb)
    ph = res["phase"]
    it_per_step = [ph["adj_iters"][k] / max(1, args.steps) for k in range(2)]
    cpu = None
    if not args.no_cpu_baseline:
        v, spent, desc = oracle_sample(wl, res["steps"], res["W"], it_per_step,
                                       collision=args.collision)
        cpu = {"value": v, "unit": "MLUPS", "cores": 1, "kind": "oracle", "sample": desc,
               "seconds": round(spent, 1)}
    line = {
        "metric": "primal/adjoint MLUPS (whole job) and % HBM roofline",
        "value": res["value"], "unit": "MLUPS", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": res["ms"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if rb == 4 else "f64",
        "data": "synthetic",
        "config": {"workload": wl.name, "grid": list(wl.dims),
                   "lattice": f"D{2 if wl.q == 9 else 3}Q{wl.q}", "storage": wl.storage,
                   "collision": args.collision, "Re": wl.Re, "u0": wl.u0, "primal_steps": res["steps"],
                   "avg_window": res["W"], "objectives": ["drag_ffa", "dissipation"],
                   "adjoint": {"mode": args.adjoint_mode, "tau_adj": args.tau_adj or None,
                               "solver": args.adjoint_solver,
                               "tol": args.adjoint_tol,
                               "max_iter": args.adjoint_max_iter,
                               "iters_per_step": it_per_step},
                   "l2": "flushed between timed steps (252 MB write)",
                   "parallelism": f"replicas{args.gpus}"},
        "roofline": roof, "cpu_baseline": cpu, "e2e": res["e2e"],
        "gpu_launches": res["launches"], "clocks": res["clocks"],
        "gradients_per_s": 2 * args.steps / (res["ms"] * 1e-3),
        "J": {"drag_ffa": res["Js"][0], "dissipation": res["Js"][1]},
    }
    print(json.dumps(line))


if __name__ == "__main__":
    main()
