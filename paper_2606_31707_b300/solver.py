"""Convenience wrapper over the C ABI: one object per context.

Still marshalling only -- it converts numpy/torch inputs to the canonical
layout of the ABI (component-major, x fastest) and back.  Shapes on the
Python side are (nz, ny, nx) for scalars and (q or dim, nz, ny, nx) for
multi-component fields.
"""
from __future__ import annotations

from typing import Optional, Sequence

import numpy as np

from . import hlbm as H


class Solver:
    """One HLBM context: primal with averages, adjoint, gradient."""

    def __init__(self, lattice: int, dims: Sequence[int], tau: float, Cs: float = 0.0,
                 storage: int = H.FP32, u_in: float = 0.05, regions=None,
                 objectives: int = H.OBJ_DRAG_FFA | H.OBJ_DISSIPATION, tau_adj: float = 0.0,
                 accum_stride: int = 1, check_every: int = 100, stream=None,
                 u_solid=(0.0, 0.0, 0.0), average_full_f: bool = False,
                 adjoint_solver: int = 0, gmres_restart: int = 30, gmres_inner: int = 100,
                 collision: int = H.COLL_BGK, inflow_profile=None, block_x: int = 0,
                 adjoint_warm_start: bool = False):
        self.q = lattice
        self.dims = tuple(int(v) for v in dims)
        self.dim = 2 if lattice == 9 else 3
        opt = self._options(storage, u_in, regions, objectives, tau_adj, accum_stride,
                            check_every, u_solid, average_full_f)
        opt.adjoint_solver = adjoint_solver
        opt.gmres_restart = gmres_restart
        opt.gmres_inner = gmres_inner
        opt.collision = collision
        opt.block_x = block_x
        opt.adjoint_warm_start = int(adjoint_warm_start)
        prof = None
        if inflow_profile is not None:
            prof = np.ascontiguousarray(inflow_profile, dtype=np.float64).ravel()
            if prof.size != self.dims[1] * self.dims[2]:
                raise ValueError("inflow_profile needs ny * nz values")
            opt.inflow_ux = prof.ctypes.data
        if stream is not None:
            opt.stream = stream if isinstance(stream, int) else int(stream.cuda_stream)
        self.opt = opt
        # bumped by every call that changes the state or the averages, so that a
        # pending autograd backward can tell its forward's state was replaced
        self.generation = 0
        self.last_adjoint = None
        self.ctx = H.hlbm_create(lattice, self.dims, tau, Cs, opt)
        opt.inflow_ux = None  # copied by the library
        self.xi, self.w = H.hlbm_velocity_set(lattice)
        self._design(opt)

    def _options(self, storage, u_in, regions, objectives, tau_adj, accum_stride, check_every,
                 u_solid, average_full_f):
        opt = H.hlbm_default_options(self.dims)
        opt.storage = storage
        opt.u_in = u_in
        for k in range(3):
            opt.u_solid[k] = u_solid[k]
        opt.tau_adj = tau_adj
        opt.objectives = objectives
        opt.accum_stride = accum_stride
        opt.check_every = check_every
        opt.average_full_f = int(average_full_f)
        if regions is not None:
            opt.ffa_x = regions.ffa_x
            opt.ffa_y0, opt.ffa_y1 = regions.ffa_y
            opt.ffa_z0, opt.ffa_z1 = regions.ffa_z
            for k in range(6):
                opt.diss_box[k] = regions.diss_box[k]
                opt.design_box[k] = regions.design_box[k]
        return opt

    def _design(self, opt):
        box = list(opt.design_box)
        self.design_shape = (box[5] - box[4], box[3] - box[2], box[1] - box[0])

    def configure(self, tau: float, Cs: float = 0.0, u_in: float = 0.05, regions=None,
                  objectives: int = H.OBJ_DRAG_FFA | H.OBJ_DISSIPATION, tau_adj: float = 0.0,
                  accum_stride: int = 1, check_every: int = 100, u_solid=(0.0, 0.0, 0.0),
                  average_full_f: bool = False, adjoint_solver: int = 0, gmres_restart: int = 30,
                  gmres_inner: int = 100, inflow_profile=None, adjoint_warm_start: bool = False):
        """New physical parameters for this context (same grid and storage)."""
        opt = self._options(self.opt.storage, u_in, regions, objectives, tau_adj, accum_stride,
                            check_every, u_solid, average_full_f)
        opt.adjoint_solver = adjoint_solver
        opt.gmres_restart = gmres_restart
        opt.gmres_inner = gmres_inner
        opt.collision = self.opt.collision
        opt.adjoint_warm_start = int(adjoint_warm_start)
        prof = None
        if inflow_profile is not None:
            prof = np.ascontiguousarray(inflow_profile, dtype=np.float64).ravel()
            if prof.size != self.dims[1] * self.dims[2]:
                raise ValueError("inflow_profile needs ny * nz values")
            opt.inflow_ux = prof.ctypes.data
        H.hlbm_configure(self.ctx, tau, Cs, opt)
        self.generation += 1
        opt.inflow_ux = None
        self._design(opt)

    # ------------------------------------------------------------------
    @property
    def shape(self):
        nx, ny, nz = self.dims
        return (nz, ny, nx)

    def set_porosity(self, d):
        self.generation += 1
        H.hlbm_set_porosity(self.ctx, np.ascontiguousarray(d, dtype=np.float64).ravel()
                            if isinstance(d, np.ndarray) else d)

    def init_equilibrium(self, rho=None, u=None):
        if u is not None and isinstance(u, np.ndarray):
            u = np.ascontiguousarray(u[: self.dim], dtype=np.float64)
        if rho is not None and isinstance(rho, np.ndarray):
            rho = np.ascontiguousarray(rho, dtype=np.float64)
        self.generation += 1
        H.hlbm_init_equilibrium(self.ctx, rho, u)

    def run_primal(self, steps: int, avg_window: int = 0):
        self.generation += 1
        return H.hlbm_run_primal(self.ctx, steps, avg_window)

    def objective(self, obj: int) -> float:
        return H.hlbm_objective(self.ctx, obj)

    def solve_adjoint(self, obj: int, mode: int = H.ADJ_EXACT, tol: float = 1e-8,
                      max_iter: int = 100000):
        return H.hlbm_solve_adjoint(self.ctx, obj, mode, tol, max_iter)

    def gradient(self, out=None):
        if out is None:
            out = np.empty(self.design_shape, dtype=np.float64)
        H.hlbm_gradient(self.ctx, out)
        return out

    _NCOMP = {H.FIELD_RHO: 1, H.FIELD_U: None, H.FIELD_F: "q", H.FIELD_FBAR: "q",
              H.FIELD_GBAR_FFA: "q", H.FIELD_GBAR_DISS: "q", H.FIELD_DJDD_FFA: 1,
              H.FIELD_DJDD_DISS: 1, H.FIELD_TAU_T: 1, H.FIELD_LAMBDA: "q",
              H.FIELD_POROSITY: 1}

    def _ncomp(self, which):
        n = self._NCOMP[which]
        if n == "q":
            return self.q
        if n is None:
            return self.dim
        return n

    def field(self, which: int):
        n = self._ncomp(which)
        out = np.empty((n,) + self.shape if n > 1 else self.shape, dtype=np.float64)
        H.hlbm_get_field(self.ctx, which, out)
        return out

    def set_field(self, which: int, data):
        self.generation += 1
        H.hlbm_set_field(self.ctx, which, np.ascontiguousarray(data, dtype=np.float64)
                         if isinstance(data, np.ndarray) else data)

    def stats(self):
        return H.hlbm_get_stats(self.ctx)

    def save(self, path):
        H.hlbm_save(self.ctx, path)

    def load(self, path):
        self.generation += 1
        H.hlbm_load(self.ctx, path)

    def close(self):
        if getattr(self, "ctx", None) is not None:
            H.hlbm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
