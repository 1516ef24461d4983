"""Continuous-batching server for mean-flow sensitivity requests.

A request is one whole Algorithm-1 solve (primal with averages, adjoint,
gradient) on its own grid and porosity field.  The server keeps a fixed
number of slots; a request is admitted as soon as a slot is free and its
device footprint fits the HBM budget, so requests that arrive while others
run join immediately and their kernels overlap on the GPU (each slot owns a
context and a CUDA stream, driven by its own host thread; the C ABI releases
the GIL).  All state of a request stays on the device until its gradient is
copied out.  Every reduction in the library is per request and in a fixed
order, so a result does not depend on what else is running.  A request marked
``warm_start`` that lands on a pooled context starts its adjoint from the
previous request's adjoint on that context (the same fixed point and
stopping rule, from a nearby start); its result then matches a cold solve
within the request's tolerance rather than bitwise.

This module is orchestration only: every arithmetic step runs in the CUDA
library.
"""
from __future__ import annotations

import queue
import threading
import time
from concurrent.futures import Future
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np

from . import hlbm as H
from .solver import Solver


@dataclass
class Request:
    q: int
    dims: Sequence[int]
    tau: float
    porosity: np.ndarray                 # (nz, ny, nx)
    u_in: float = 0.05
    Cs: float = 0.0
    warm_steps: int = 2000
    avg_steps: int = 2000
    objective: int = H.OBJ_DRAG_FFA
    mode: int = H.ADJ_EXACT
    tol: float = 1e-6
    max_iter: int = 4000
    storage: int = H.FP32
    regions: object = None
    tag: object = None
    t_submit: float = 0.0
    adjoint_solver: int = 0              # 0 fixed point, 1 restarted GMRES (same fixed point)
    gmres_restart: int = 30
    gmres_inner: int = 100               # sweep pairs per Krylov operator application
    warm_start: bool = False             # on a reused context, start the adjoint from the
                                         # previous request's (same fixed point and tolerance)
    block_x: int = 0                     # threads per block along x (0: chosen by grid size)


@dataclass
class Result:
    tag: object
    J: float
    gradient: np.ndarray
    adjoint_iters: int
    adjoint_residual: float
    status: int
    latency_s: float
    queued_s: float
    lups: int


def footprint_bytes(q: int, dims: Sequence[int], storage: int = H.FP32, objectives: int = 1,
                    adjoint_solver: int = 0, gmres_restart: int = 30) -> int:
    """Device bytes one request holds (populations, averages, adjoint state,
    and the Krylov basis when the adjoint runs GMRES)."""
    nx, ny, nz = dims
    N = nx * ny * nz
    pop = {H.FP64: 8, H.FP32: 4, H.FP16DEV: 2, H.BF16DEV: 2}[storage]
    real = 8 if storage == H.FP64 else 4
    D = 2 if q == 9 else 3
    b = q * N * pop + N * real                       # populations, porosity
    b += q * N * 8 + N * 8                           # sum f, sum tau
    b += objectives * (q * N * 8 + N * 8)            # sum dJ/df, dJ/dd
    b += 2 * q * N * real + q * N * real + (D + 2) * N * real  # lambda, snapshot, source, record
    b += q * N * 8 * 2                               # staging for readouts
    if adjoint_solver == 1:
        b += (gmres_restart + 4) * q * N * real      # basis, w, x, c
    return int(b)


class ContextPool:
    """Idle contexts kept for reuse, keyed by (lattice, grid, storage).

    Reusing a context avoids its allocations and frees (cudaFree waits for the
    whole device, which would stall every other request in flight) and keeps
    its captured CUDA graphs.  Idle contexts count against the HBM budget and
    are destroyed, oldest first, when an admission needs their memory."""

    def __init__(self):
        self._idle = {}          # key -> list of (Solver, bytes)
        self._order: List[tuple] = []
        self.idle_bytes = 0
        self.hits = 0
        self.misses = 0

    def take(self, key):
        lst = self._idle.get(key)
        if lst:
            s, b = lst.pop()
            self._order.remove((key, id(s)))
            self.idle_bytes -= b
            self.hits += 1
            return s
        self.misses += 1
        return None

    def give(self, key, solver, nbytes):
        self._idle.setdefault(key, []).append((solver, nbytes))
        self._order.append((key, id(solver)))
        self.idle_bytes += nbytes

    def evict_one(self) -> bool:
        if not self._order:
            return False
        key, sid = self._order.pop(0)
        lst = self._idle[key]
        for k, (s, b) in enumerate(lst):
            if id(s) == sid:
                lst.pop(k)
                self.idle_bytes -= b
                s.close()
                return True
        return False

    def clear(self):
        while self.evict_one():
            pass


def _key(req: "Request"):
    return (req.q, tuple(req.dims), req.storage)


BATCH_BLOCK_X = 128  # the block width batched contexts share (the library's NT)


def batchable(req: "Request", max_cells: int) -> bool:
    """Requests the batched lane can step together: FP32, BGK without the
    Smagorinsky model, the fixed-point adjoint, J_FFA or J_DISS, and a grid
    small enough that it cannot fill the GPU alone."""
    return (req.storage == H.FP32 and req.Cs == 0.0 and req.adjoint_solver == 0
            and req.objective in (H.OBJ_DRAG_FFA, H.OBJ_DISSIPATION)
            and int(np.prod(req.dims)) <= max_cells)


class SensitivityServer:
    """Admit requests into at most ``slots`` concurrent solves within
    ``hbm_budget`` bytes; results are returned through futures.

    Requests that ``batchable`` accepts (grids of at most ``batch_cells``
    cells) go to the batched lane instead: one host thread takes every such
    request waiting, up to ``batch_slots``, as a cohort and steps them together
    on one stream through the library's batched entry points (one kernel launch
    per primal step or adjoint sweep for the whole cohort), while the other
    requests run concurrently on their own contexts and streams.  Requests
    that arrive while a cohort runs form the next one."""

    def __init__(self, slots: int = 8, hbm_budget: int = 200 << 30, reuse_contexts: bool = True,
                 batch_cells: int = 400_000, batch_slots: int = 32):
        self.slots = slots
        self.budget = hbm_budget
        self.batch_cells = batch_cells
        self.batch_slots = batch_slots
        self._bpending: List[tuple] = []
        self.cohorts: List[int] = []
        self._q: "queue.Queue[tuple]" = queue.Queue()
        self._used = 0
        self._active = 0
        self._cv = threading.Condition()
        self._stop = False
        self._threads: List[threading.Thread] = []
        self._sched = threading.Thread(target=self._schedule, daemon=True)
        self._pending: List[tuple] = []
        self.completed: List[Result] = []
        self.pool = ContextPool() if reuse_contexts else None
        self._sched.start()
        self._batch_thread = None
        if batch_cells > 0:
            self._batch_thread = threading.Thread(target=self._batch_loop, daemon=True)
            self._batch_thread.start()

    # ------------------------------------------------------------------
    def submit(self, req: Request) -> Future:
        fut: Future = Future()
        req.t_submit = time.perf_counter()
        need = footprint_bytes(req.q, req.dims, req.storage, adjoint_solver=req.adjoint_solver,
                               gmres_restart=req.gmres_restart)
        if need > self.budget:
            fut.set_exception(H.HlbmError(H.ENOMEM, "request larger than the HBM budget"))
            return fut
        with self._cv:
            if self._batch_thread is not None and batchable(req, self.batch_cells):
                self._bpending.append((req, fut, need))
            else:
                self._pending.append((req, fut, need))
            self._cv.notify_all()
        return fut

    def close(self):
        with self._cv:
            self._stop = True
            self._cv.notify_all()
        self._sched.join()
        if self._batch_thread is not None:
            self._batch_thread.join()
        for t in self._threads:
            t.join()
        if self.pool is not None:
            self.pool.clear()

    # ------------------------------------------------------------------
    def _schedule(self):
        while True:
            with self._cv:
                while not self._stop and not self._admissible():
                    self._cv.wait(timeout=0.05)
                if self._stop and not self._pending:
                    return
                if not self._admissible():
                    continue
                # first-come first-served among requests that fit; a reusable idle
                # context of the same shape needs no new memory
                k = next(i for i, (_, _, need) in enumerate(self._pending)
                         if self._fits(need))
                req, fut, need = self._pending.pop(k)
                solver = self.pool.take(_key(req)) if self.pool is not None else None
                if solver is not None:
                    # a reused context keeps every buffer it ever allocated (a
                    # Krylov basis of an earlier GMRES request, for instance):
                    # account for the most it has held
                    need = max(need, getattr(solver, "held_bytes", need))
                else:
                    while self.pool is not None and self._used + self.pool.idle_bytes + need > self.budget:
                        if not self.pool.evict_one():
                            break
                self._used += need
                self._active += 1
            t = threading.Thread(target=self._run, args=(req, fut, need, solver), daemon=True)
            t.start()
            self._threads.append(t)

    # ------------------------------------------------------------------
    def _batch_loop(self):
        import torch

        stream = torch.cuda.Stream()
        sptr = int(stream.cuda_stream)
        batches = {}
        idle = {}   # (q, dims) -> idle Solvers of this lane (created on its stream)
        while True:
            with self._cv:
                while not self._stop and not self._batch_admissible():
                    self._cv.wait(timeout=0.05)
                if self._stop and not self._bpending:
                    break
                cohort = []
                rest = []
                for item in self._bpending:
                    if len(cohort) < self.batch_slots and self._fits(item[2]):
                        cohort.append(item)
                        self._used += item[2]
                    else:
                        rest.append(item)
                self._bpending = rest
            if not cohort:
                continue
            self.cohorts.append(len(cohort))
            groups = {}
            for item in cohort:
                r = item[0]
                groups.setdefault((r.q, r.warm_steps, r.avg_steps, r.mode, r.tol, r.max_iter),
                                  []).append(item)
            for key, items in groups.items():
                q = key[0]
                if q not in batches:
                    batches[q] = H.hlbm_batch_create(q, sptr)
                self._run_cohort(batches[q], items, idle, sptr)
            with self._cv:
                for _, _, need in cohort:
                    self._used -= need
                self._cv.notify_all()
        for b in batches.values():
            H.hlbm_batch_destroy(b)
        for lst in idle.values():
            for s_ in lst:
                s_.close()

    def _run_cohort(self, batch, items, idle, sptr):
        t0 = time.perf_counter()
        solvers = []
        try:
            for req, _, _ in items:
                key = (req.q, tuple(req.dims))
                s_ = idle[key].pop() if idle.get(key) else None
                if s_ is None:
                    s_ = Solver(req.q, req.dims, req.tau, req.Cs, storage=H.FP32, u_in=req.u_in,
                                regions=req.regions, objectives=req.objective, stream=sptr,
                                block_x=BATCH_BLOCK_X)
                else:
                    s_.configure(req.tau, req.Cs, u_in=req.u_in, regions=req.regions,
                                 objectives=req.objective)
                solvers.append(s_)
                s_.set_porosity(req.porosity)
                H.hlbm_init_equilibrium(s_.ctx)
            ctxs = [s_.ctx for s_ in solvers]
            r0 = items[0][0]
            steps = r0.warm_steps + r0.avg_steps
            H.hlbm_batch_run_primal(batch, ctxs, steps, r0.avg_steps)
            Js = [s_.objective(req.objective) for s_, (req, _, _) in zip(solvers, items)]
            _, per = H.hlbm_batch_solve_adjoint(batch, ctxs, [req.objective for req, _, _ in items],
                                                r0.mode, r0.tol, r0.max_iter)
            for s_, (req, fut, _), J, (st, it, res) in zip(solvers, items, Js, per):
                if st < 0:
                    fut.set_exception(H.HlbmError(st, H.hlbm_last_error(s_.ctx)))
                    continue
                G = s_.gradient()
                N = int(np.prod(req.dims))
                out = Result(req.tag, J, G, it, res, st, 0.0, 0.0, N * (steps + it))
                out.queued_s = t0 - req.t_submit
                out.latency_s = time.perf_counter() - req.t_submit
                self.completed.append(out)
                fut.set_result(out)
        except Exception as e:  # noqa: BLE001 - forwarded to the callers
            for _, fut, _ in items:
                if not fut.done():
                    fut.set_exception(e)
        finally:
            for s_, (req, _, _) in zip(solvers, items):
                idle.setdefault((req.q, tuple(req.dims)), []).append(s_)

    def _batch_admissible(self) -> bool:
        return any(self._fits(need) for _, _, need in self._bpending)

    def _fits(self, need: int) -> bool:
        # idle pooled contexts can always be evicted to make room
        return self._used + need <= self.budget

    def _admissible(self) -> bool:
        if self._active >= self.slots or not self._pending:
            return False
        return any(self._fits(need) for _, _, need in self._pending)

    def _run(self, req: Request, fut: Future, need: int, solver):
        t0 = time.perf_counter()
        keep = None
        try:
            res, keep = solve_one(req, solver, keep_context=self.pool is not None)
            res.queued_s = t0 - req.t_submit
            res.latency_s = time.perf_counter() - req.t_submit
            self.completed.append(res)
            fut.set_result(res)
        except Exception as e:  # noqa: BLE001 - forwarded to the caller
            fut.set_exception(e)
        finally:
            with self._cv:
                self._used -= need
                self._active -= 1
                if keep is not None:
                    keep.held_bytes = max(need, getattr(keep, "held_bytes", 0))
                    self.pool.give(_key(req), keep, keep.held_bytes)
                self._cv.notify_all()


def solve_one(req: Request, solver: Optional[Solver] = None, keep_context: bool = False):
    """Algorithm 1 for one request on its own context and stream.

    With ``solver`` an idle context of the same grid and storage is reused
    (reconfigured for the request).  Returns the Result, and with
    ``keep_context`` also the context (else it is destroyed)."""
    if solver is None:
        s = Solver(req.q, req.dims, req.tau, req.Cs, storage=req.storage, u_in=req.u_in,
                   regions=req.regions, objectives=req.objective,
                   adjoint_solver=req.adjoint_solver, gmres_restart=req.gmres_restart,
                   gmres_inner=req.gmres_inner, block_x=req.block_x)
    else:
        s = solver
        s.configure(req.tau, req.Cs, u_in=req.u_in, regions=req.regions, objectives=req.objective,
                    adjoint_solver=req.adjoint_solver, gmres_restart=req.gmres_restart,
                    gmres_inner=req.gmres_inner, adjoint_warm_start=req.warm_start)
    ok = False
    try:
        s.set_porosity(req.porosity)
        H.hlbm_init_equilibrium(s.ctx)
        steps = req.warm_steps + req.avg_steps
        s.run_primal(steps, req.avg_steps)
        J = s.objective(req.objective)
        st, it, res = s.solve_adjoint(req.objective, req.mode, req.tol, req.max_iter)
        G = s.gradient()
        N = int(np.prod(req.dims))
        ok = True
        result = Result(req.tag, J, G, it, res, st, 0.0, 0.0, N * (steps + it))
    finally:
        if not (ok and keep_context):
            s.close()
    if keep_context:
        return result, s
    return result
