"""Benchmark of the HLBM mean-flow adjoint hot path on B300.

Workload (default): the LES cylinder case, D3Q19 640x320x100 (20.48 M cells),
BGK with the Smagorinsky relaxation time (C_S = 0.1), Re 3900, u0 0.05,
FP32 populations -- the largest single-GPU configuration.  Its whole job
(32 000 warm-up steps, 32 000 averaged steps, adjoints to convergence) takes
minutes, so one benchmark step is a fixed slice of Algorithm 1 on the full
grid, continuing the flow from the previous step:

  porosity upload, P plain primal steps, a tracking window of W averaged
  steps (f, J, dJ/df, dJ/dd, tau_eff - tau0), then for the drag (J_FFA) and
  the dissipation (J_DISS) objectives: the linearisation at the window's
  mean, M adjoint sweeps of the fixed-point iteration from zero for each
  (tolerance 0: a fixed sweep count, so the status is NOT_CONVERGED by
  construction and is reported with the residual) and the gradient.

value = lattice updates of the slice (N x (P + W + 2 M)) per second on the
device, inputs resident; e2e = the same through the C ABI with host buffers
(porosity uploaded, both gradients downloaded every step).  After the timed
regions, untimed: the gradient of the last slice against a GMRES solve of
the same fixed point (the accuracy the slice's sweep count gives), and the
sweeps and time GMRES needs to reach its tolerance.  roofline: the dominant
kernel against the measured HBM copy bandwidth.  cpu_baseline: the FP64
oracle on a bounded sub-box of the same workload, one thread and all host
cores (one process per core).

``--impl reference`` times the oracle itself (the only reference there is)
on the host cores, for the same workload, slice and metric.
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
# its capture reports traffic null.  The ncu summaries sit under profiles/.
MEASURED_DRAM = {
    # captured on the 640x320x24 slab of the LES grid (the same x-y plane, 4.9 M
    # cells, the same bytes per update to 0.01 %) and scaled to the 640x320x100
    # grid by the cell ratio 100 / 24; captured at sources 6e82031b298c54da, which
    # differ from these only in a comment
    ("5c3e4eafdeb3c81c", "les3d_re3900", "fp32", "bgk", "primal_step_accumulate"): 7_779_937_067,
    ("5c3e4eafdeb3c81c", "les3d_re3900", "fp32", "bgk", "primal_step_plain"): 2_960_550_933,
    ("5c3e4eafdeb3c81c", "les3d_re3900", "fp32", "bgk", "adjoint_step_ffa"): 4_613_611_200,
    ("5c3e4eafdeb3c81c", "les3d_re3900", "fp32", "bgk", "adjoint_step_diss"): 5_293_752_533,
    ("5c3e4eafdeb3c81c", "les3d_re3900_slab", "fp32", "bgk", "primal_step_accumulate"): 1_867_184_896,
    ("5c3e4eafdeb3c81c", "les3d_re3900_slab", "fp32", "bgk", "primal_step_plain"): 710_532_224,
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
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="les3d_re3900")
    ap.add_argument("--setup-steps", type=int, default=4096,
                    help="untimed plain steps that develop the flow before the first step")
    ap.add_argument("--slice-plain", type=int, default=64, help="plain primal steps per step (P)")
    ap.add_argument("--slice-avg", type=int, default=64, help="averaged primal steps per step (W)")
    ap.add_argument("--slice-sweeps", type=int, default=64,
                    help="adjoint sweeps per objective and step (M)")
    ap.add_argument("--adjoint-mode", default="exact", choices=["exact", "fta"])
    ap.add_argument("--tau-adj", type=float, default=None,
                    help="adjoint relaxation time, the regularisation of Sec. 5.4 "
                         "(default: 0.6, the paper's LES setting, when C_S > 0, else tau0)")
    ap.add_argument("--collision", default=None, choices=["bgk", "rr"],
                    help="BGK (Sec. 2.1) or the recursive regularised collision (Sec. 2.2); "
                         "default: the workload's (BGK)")
    ap.add_argument("--storage", default=None, choices=["fp64", "fp32", "fp16dev", "bf16dev"],
                    help="population storage (default: the workload's)")
    ap.add_argument("--reference-tol", type=float, default=1e-4,
                    help="GMRES tolerance of the untimed accuracy reference")
    ap.add_argument("--reference-max-sweeps", type=int, default=40000)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-procs", type=int, default=None,
                    help="oracle processes of the all-core CPU figures (default: host cores, "
                         "at most 32)")
    return ap.parse_args()


def resolve(args, wl):
    """Fill the workload-dependent defaults into args."""
    if args.collision is None:
        args.collision = wl.collision
    if args.tau_adj is None:
        args.tau_adj = 0.6 if wl.Cs > 0 else 0.0
    return args


def storage_code(H, wl):
    return {"fp64": H.FP64, "fp32": H.FP32, "fp16dev": H.FP16DEV, "bf16dev": H.BF16DEV}[wl.storage]


# ---------------------------------------------------------------------------
# algorithmic bytes per lattice update
# ---------------------------------------------------------------------------

def bytes_model(wl, storage_bytes, real_bytes, exact_rec=False, rr=False):
    """Algorithmic bytes per lattice update of each kernel (reads + writes).

    Averaging step: the populations and porosity of a plain step plus, for
    each running sum it updates, a read-modify-write of the sum -- 16 B for
    FP64 storage; for the other storages the sample goes to a float staging
    value (8 B) that is folded into the FP64 sum every 64 samples
    (16 B + 8 B, amortised 0.375 B).  Sums: the averaged state -- all q
    populations when f_bar itself is needed (the exact LES linearisation of
    BGK), else its moments (rho - 1 and rho u, plus the D(D+1)/2 second
    moments for the regularised collision) -- and tau_eff - tau0 when
    Cs > 0; inside the objective regions the dJ/df coefficients (2 on the
    drag plane, 1 + D + D(D+1)/2 in the dissipation box) and dJ/dd.  The
    regularised collision's adjoint record is rho, u, omega and the stress
    (2 + D + D(D+1)/2 planes)."""
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
    full = les and not rr
    state = q if full else 1 + D + (D * (D + 1) // 2 if rr else 0)
    acc = plain + sb * (state + (1 if les else 0))
    acc += (ffa_cells * sb * 2 + diss_cells * sb * (1 + D + D * (D + 1) // 2 + 1)) / N
    rec = D + 2 + D * (D + 1) // 2 if rr else (q if exact_rec else D + 2)
    # the source: the derivative polynomial's coefficients in the objective's region
    adj_ffa = (2 * q + rec + 1) * real_bytes + ffa_cells * 2 * real_bytes / N
    adj_diss = (2 * q + rec + 1) * real_bytes + diss_cells * (1 + D + D * (D + 1) // 2) * real_bytes / N
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




METRIC = "primal/adjoint MLUPS and % HBM roofline"
STATUS = {0: "OK", 1: "NOT_CONVERGED", -5: "ENONFINITE", -6: "EDIVERGED"}


def run_ours(args, rank, world):
    import dataclasses

    import torch

    from paper_2606_31707_b300 import Solver
    from paper_2606_31707_b300 import hlbm as H

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    wl = make_workload(args.workload, seed=rank)
    if args.storage:
        wl = dataclasses.replace(wl, storage=args.storage)
    resolve(args, wl)
    Pn, Wn, M = args.slice_plain, args.slice_avg, args.slice_sweeps
    stream = torch.cuda.Stream(device=dev)
    coll = H.COLL_RR if args.collision == "rr" else H.COLL_BGK
    s = Solver(wl.q, wl.dims, tau_of(wl), wl.Cs, storage=storage_code(H, wl), u_in=wl.u0,
               regions=wl.regions, stream=stream, tau_adj=args.tau_adj, collision=coll)
    mode = H.ADJ_EXACT if args.adjoint_mode == "exact" else H.ADJ_FTA
    N = wl.cells
    D = 2 if wl.q == 9 else 3
    d_host = torch.from_numpy(np.ascontiguousarray(wl.porosity.ravel())).pin_memory()
    d_dev = d_host.to(dev)
    up = wl.u_perturb if wl.u_perturb is not None else np.zeros((3,) + wl.porosity.shape)
    u0 = up.copy()
    u0[0] += wl.u0
    u_dev = torch.from_numpy(np.ascontiguousarray(u0[:D].reshape(D, -1))).to(dev)
    # untimed: the flow develops from the perturbed inflow state
    s.set_porosity(d_dev)
    H.hlbm_init_equilibrium(s.ctx, None, u_dev)
    del u_dev
    if args.setup_steps > 0:
        s.run_primal(args.setup_steps + args.setup_steps % 2, 0)
    b = wl.regions.design_box
    gvol = (b[1] - b[0]) * (b[3] - b[2]) * (b[5] - b[4])
    g_dev = torch.empty((2, gvol), dtype=torch.float64, device=dev)
    g_host = torch.empty((2, gvol), dtype=torch.float64).pin_memory()
    flush = torch.empty(int(2 * L2_BYTES // 4), dtype=torch.float32, device=dev)
    objectives = (H.OBJ_DRAG_FFA, H.OBJ_DISSIPATION)
    last = [None, None]

    def zero_phase():
        return dict(plain_ms=0.0, plain_launch=0, acc_ms=0.0, acc_launch=0, adj_ms=[0.0, 0.0],
                    adj_launch=[0, 0], adj_iters=[0, 0])

    phase = zero_phase()

    def one_step(host: bool, record: bool):
        s.set_porosity(d_host if host else d_dev)
        s.run_primal(Pn, 0)
        st = s.stats()
        if record:
            phase["plain_ms"] += st.primal_ms
            phase["plain_launch"] += st.primal_launches
        s.run_primal(Wn, Wn)
        st = s.stats()
        if record:
            phase["acc_ms"] += st.primal_ms
            phase["acc_launch"] += st.primal_launches
        lups = (Pn + Wn) * N
        Js = [s.objective(o) for o in objectives]
        for k, o in enumerate(objectives):
            status, it, res = s.solve_adjoint(o, mode, 0.0, M)
            last[k] = (status, it, res)
            st = s.stats()
            if record:
                phase["adj_ms"][k] += st.adjoint_ms
                phase["adj_launch"][k] += st.adjoint_launches
                phase["adj_iters"][k] += it
            lups += it * N
            H.hlbm_gradient(s.ctx, g_host[k] if host else g_dev[k])
        return lups, Js

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    def timed(host: bool):
        nonlocal phase
        for _ in range(args.warmup):
            one_step(host, False)
        phase = zero_phase()
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
            ms += wall if host else e0.elapsed_time(e1)
            total_lups += lups
        barrier()
        return total_lups, ms, s.stats().kernels_total - k0, Js

    sampler = ClockSampler(dev.index or 0)
    sampler.start()
    lups, ms, launches, Js = timed(False)
    clocks = sampler.stop()
    phase_dev = {k: (list(v) if isinstance(v, list) else v) for k, v in phase.items()}
    adj_state = [dict(status=STATUS.get(st, st), sweeps=it, residual=res) for st, it, res in last]
    ms = max_over_ranks(ms, world, dev)
    value = job_mlups(lups, ms, world)
    e2e = None
    if not args.no_e2e:
        lups_h, ms_h, _, _ = timed(True)
        ms_h = max_over_ranks(ms_h, world, dev)
        e2e = {"value": job_mlups(lups_h, ms_h, world), "unit": "MLUPS",
               "h2d_bytes_per_step": int(d_host.numel() * 8),
               "d2h_bytes_per_step": int(g_host.numel() * 8)}
    acc = None
    if not args.no_accuracy and rank == 0:
        acc = gradient_accuracy(args, wl, s, H, Solver, mode, coll, stream, d_dev, torch, dev)
    s.close()
    return dict(wl=wl, value=value, ms=ms, lups=lups, e2e=e2e, launches=launches,
                phase=phase_dev, clocks=clocks, Js=Js, adjoint=adj_state, accuracy=acc)


def gradient_accuracy(args, wl, s, H, Solver, mode, coll, stream, d_dev, torch, dev):
    """Untimed: the drag gradient of one slice (M fixed-point sweeps from zero)
    against a GMRES solve of the same fixed point, on a second context fed the
    same averaged state through the ABI."""
    N, q = wl.cells, wl.q
    status, it, res = s.solve_adjoint(H.OBJ_DRAG_FFA, mode, 0.0, args.slice_sweeps)
    b = wl.regions.design_box
    gvol = (b[1] - b[0]) * (b[3] - b[2]) * (b[5] - b[4])
    G_slice = torch.empty(gvol, dtype=torch.float64, device=dev)
    H.hlbm_gradient(s.ctx, G_slice)
    r = Solver(q, wl.dims, tau_of(wl), wl.Cs, storage=storage_code(H, wl), u_in=wl.u0,
               regions=wl.regions, stream=stream, tau_adj=args.tau_adj, collision=coll,
               adjoint_solver=1, gmres_restart=30, gmres_inner=100)
    r.set_porosity(d_dev)
    buf = torch.empty(q * N, dtype=torch.float64, device=dev)
    for fld, n in ((H.FIELD_FBAR, q * N), (H.FIELD_GBAR_FFA, q * N), (H.FIELD_DJDD_FFA, N),
                   (H.FIELD_TAU_T, N)):
        H.hlbm_get_field(s.ctx, fld, buf[:n])
        H.hlbm_set_field(r.ctx, fld, buf[:n])
    del buf
    t0 = time.perf_counter()
    rst, rit, rres = r.solve_adjoint(H.OBJ_DRAG_FFA, mode, args.reference_tol,
                                     args.reference_max_sweeps)
    wall = time.perf_counter() - t0
    ref_ms = r.stats().adjoint_ms
    G_ref = torch.empty(gvol, dtype=torch.float64, device=dev)
    H.hlbm_gradient(r.ctx, G_ref)
    r.close()
    err = float(torch.linalg.vector_norm(G_slice - G_ref) / torch.linalg.vector_norm(G_ref))
    return {"objective": "drag_ffa", "slice": {"solver": "fixed-point", "sweeps": it,
                                               "status": STATUS.get(status, status),
                                               "residual": res},
            "reference": {"solver": "gmres(30), 100 sweep pairs per operator", "tol": args.reference_tol,
                          "sweeps": rit, "status": STATUS.get(rst, rst), "residual": rres,
                          "gpu_s": round(ref_ms * 1e-3, 2), "wall_s": round(wall, 2)},
            "slice_gradient_rel_l2_vs_reference": err}


def roofline_of(res, args, storage_bytes, real_bytes):
    wl = res["wl"]
    N = wl.cells
    bm = bytes_model(wl, storage_bytes, real_bytes,
                     exact_rec=(wl.Cs > 0 and args.adjoint_mode == "exact"),
                     rr=args.collision == "rr")
    ph = res["phase"]
    cand = []  # (kernel, ms, launches, bytes per cell and launch)
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
            "phase_mlups": {c[0]: round(N * c[2] / (c[1] * 1e-3) / 1e6, 1) for c in cand},
            "phase_gbs": {c[0]: round(N * c[2] * c[3] / (c[1] * 1e-3) / 1e9, 1) for c in cand}}


# ---------------------------------------------------------------------------
# the oracle on a bounded sample (cpu_baseline and --impl reference)
# ---------------------------------------------------------------------------

def sample_box(wl):
    """A sub-box of the workload around the front of its body: (x0, x1, y0, y1, z0, z1)."""
    nx, ny, nz = wl.dims
    if wl.q == 19:
        w, h, t = 48, 24, 16
    else:
        w, h, t = 96, 48, 1
    w, h, t = min(w, nx), min(h, ny), min(t, nz)
    x0 = max(0, min(nx - w, int(wl.regions.ffa_x) - w - 40)) if nx > w else 0
    y0 = max(0, (ny - h) // 2)
    return (x0, x0 + w, y0, y0 + h, 0, t)


def sample_inputs(wl):
    """The sub-box's porosity and initial velocity perturbation (small arrays)."""
    x0, x1, y0, y1, z0, z1 = sample_box(wl)
    d = np.ascontiguousarray(wl.porosity[z0:z1, y0:y1, x0:x1])
    up = None if wl.u_perturb is None else np.ascontiguousarray(wl.u_perturb[:, z0:z1, y0:y1, x0:x1])
    return d, up


def oracle_sample(q, u0, L, Re, Cs, d, up, collision, mode, tau_adj, Pn, Wn, M,
                  n_plain=2, n_acc=1, n_adj=2):
    """Time the FP64 oracle, as it stands, on a sub-box of a workload (its own
    periodic problem with inflow and outflow at the box's x faces) and return
    (MLUPS of the slice's update mix, seconds spent).  Runs in one process."""
    from oracle import adjoint as oadj
    from oracle import hlbm as ohlbm
    from oracle import meanflow as omf
    from workloads import Regions

    t_start = time.perf_counter()
    dims = (d.shape[2], d.shape[1], d.shape[0])
    P = ohlbm.Params(q, dims, tau0=ohlbm.tau_from_reynolds(u0, L, Re), Cs=Cs, u_in=u0,
                     collision=collision)
    R = Regions(ffa_x=dims[0] - 3, ffa_y=(0, dims[1]), ffa_z=(0, dims[2]),
                diss_box=(0, dims[0], 0, dims[1], 0, dims[2]),
                design_box=(0, dims[0], 0, dims[1], 0, dims[2]))
    f = ohlbm.initial_state(P, up)
    t = time.perf_counter()
    for _ in range(n_plain):
        f = ohlbm.step(f, d, P)
    t_plain = (time.perf_counter() - t) / n_plain
    t = time.perf_counter()
    out = omf.run_primal(f, d, P, n_acc, n_acc, R, 3)
    t_acc = (time.perf_counter() - t) / n_acc
    t = time.perf_counter()
    lin = oadj.Linearisation(out["fbar"], d, P, oadj.EXACT if mode == "exact" else oadj.FTA,
                             tau_adj or None, out["tau_t_bar"])
    t_lin = time.perf_counter() - t
    t = time.perf_counter()
    lam, _, _ = oadj.solve_adjoint(lin, out[("gbar", 1)], tol=0.0, max_iter=n_adj)
    t_adj = (time.perf_counter() - t) / n_adj
    t = time.perf_counter()
    oadj.gradient(lin, lam, out[("dJdd_bar", 1)])
    t_grad = time.perf_counter() - t
    n = dims[0] * dims[1] * dims[2]
    slice_s = Pn * t_plain + Wn * t_acc + 2 * (t_lin + M * t_adj + t_grad)
    return n * (Pn + Wn + 2 * M) / slice_s / 1e6, time.perf_counter() - t_start


def _sample_worker(a):
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    return oracle_sample(*a)


class OraclePool:
    """One oracle process per host core (at most ``cap``), started with spawn."""

    def __init__(self, procs):
        import multiprocessing as mp
        self.procs = procs
        self.pool = mp.get_context("spawn").Pool(procs)

    def round(self, a):
        """Every process times one sample at once; returns (summed MLUPS, wall s)."""
        t = time.perf_counter()
        res = self.pool.map(_sample_worker, [a] * self.procs)
        return sum(v for v, _ in res), time.perf_counter() - t

    def close(self):
        self.pool.close()
        self.pool.join()


def host_procs(args):
    return max(1, min(args.cpu_procs or (os.cpu_count() or 1), 32))


def sample_desc(wl, args, procs):
    b = sample_box(wl)
    return (f"FP64 oracle (numpy/scipy, as it stands) on a {b[1]-b[0]}x{b[3]-b[2]}x{b[5]-b[4]} "
            f"sub-box of the {wl.dims[0]}x{wl.dims[1]}x{wl.dims[2]} grid (its own problem: inflow "
            f"and outflow at the box faces, dissipation over the whole box): 2 plain steps, 1 "
            f"averaging step, one linearisation ({args.adjoint_mode}, tau_adj {args.tau_adj or 'tau0'}), "
            f"2 adjoint sweeps and a gradient timed, extrapolated to the slice's mix of "
            f"{args.slice_plain} plain + {args.slice_avg} averaging steps + 2 x ({args.slice_sweeps} "
            f"sweeps + linearisation + gradient); {procs} process(es) at once, one thread each")


def sample_args(wl, args):
    d, up = sample_inputs(wl)
    return (wl.q, wl.u0, wl.L, wl.Re, wl.Cs, d, up, args.collision, args.adjoint_mode,
            args.tau_adj, args.slice_plain, args.slice_avg, args.slice_sweeps)


def cpu_baseline(args, wl):
    a = sample_args(wl, args)
    v1, sec1 = oracle_sample(*a)
    procs = host_procs(args)
    pool = OraclePool(procs)
    try:
        vall, wall = pool.round(a)
    finally:
        pool.close()
    return {"value": vall, "unit": "MLUPS", "cores": procs, "kind": "oracle",
            "sample": sample_desc(wl, args, procs),
            "one_thread": {"value": v1, "unit": "MLUPS", "cores": 1, "seconds": round(sec1, 1)},
            "host_cores": os.cpu_count(), "seconds": round(sec1 + wall, 1)}


def run_reference(args):
    wl = make_workload(args.workload)
    if args.storage:
        import dataclasses
        wl = dataclasses.replace(wl, storage=args.storage)
    resolve(args, wl)
    a = sample_args(wl, args)
    procs = host_procs(args)
    pool = OraclePool(procs)
    vals = []
    try:
        for k in range(args.warmup + args.steps):
            v, wall = pool.round(a)
            if k >= args.warmup:
                vals.append((v, wall))
    finally:
        pool.close()
    value = statistics.median(v for v, _ in vals)
    ms = statistics.median(w for _, w in vals) * 1e3
    line = {"impl": "reference", "metric": METRIC, "value": value,
            "unit": "MLUPS", "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(wl, args),
            "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": procs, "kind": "oracle",
                             "sample": sample_desc(wl, args, procs)},
            "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def config_of(wl, args):
    return {"workload": wl.name, "grid": list(wl.dims), "cells": wl.cells,
            "lattice": f"D{2 if wl.q == 9 else 3}Q{wl.q}", "storage": wl.storage,
            "collision": args.collision, "Cs": wl.Cs, "Re": wl.Re, "u0": wl.u0,
            "tau0": tau_of(wl),
            "slice": {"plain_steps": args.slice_plain, "averaged_steps": args.slice_avg,
                      "adjoint_sweeps_per_objective": args.slice_sweeps,
                      "objectives": ["drag_ffa", "dissipation"]},
            "setup_steps_untimed": args.setup_steps,
            "adjoint": {"mode": args.adjoint_mode, "tau_adj": args.tau_adj or None,
                        "solver": "fixed-point", "tol": 0.0},
            "l2": (f"flushed between timed steps (252 MB write); populations alone "
                   f"{wl.q * wl.cells * {'fp64': 8, 'fp32': 4}.get(wl.storage, 2) / 1e9:.2f} GB"),
            "parallelism": f"replicas{args.gpus}"}


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
    cpu = None if args.no_cpu_baseline else cpu_baseline(args, wl)
    cfg = config_of(wl, args)
    cfg["adjoint"]["last_step"] = {"drag_ffa": res["adjoint"][0], "dissipation": res["adjoint"][1]}
    line = {
        "metric": METRIC,
        "value": res["value"], "unit": "MLUPS", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": res["ms"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if rb == 4 else "f64",
        "data": "synthetic",
        "config": cfg,
        "roofline": roof, "cpu_baseline": cpu, "e2e": res["e2e"],
        "gpu_launches": res["launches"], "clocks": res["clocks"],
        "gradient_accuracy": res["accuracy"],
        "J": {"drag_ffa": res["Js"][0], "dissipation": res["Js"][1]},
    }
    print(json.dumps(line))


if __name__ == "__main__":
    main()
