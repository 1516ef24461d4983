"""Thin ctypes binding of the C ABI in ``include/hlbm.h``.

Argument marshalling only: every step of the method runs in the CUDA kernels
of ``libhlbm.so``.  Functions keep the C names; buffers may be numpy arrays
(host) or CUDA torch tensors (device, passed by pointer on the caller's
stream semantics of the context).  A negative status raises ``HlbmError``.

The library is loaded from this package directory; if it is missing the
import fails loudly (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhlbm.so")

D2Q9, D3Q19 = 9, 19
FP64, FP32, FP16DEV, BF16DEV = 0, 1, 2, 3
OBJ_DRAG_FFA, OBJ_DISSIPATION, OBJ_DRAG_MEA = 1, 2, 4
ADJ_EXACT, ADJ_FTA = 0, 1
COLL_BGK, COLL_RR = 0, 1
DTYPE_F64, DTYPE_F32 = 0, 1
(FIELD_RHO, FIELD_U, FIELD_F, FIELD_FBAR, FIELD_GBAR_FFA, FIELD_GBAR_DISS, FIELD_DJDD_FFA,
 FIELD_DJDD_DISS, FIELD_TAU_T, FIELD_LAMBDA, FIELD_POROSITY) = range(11)
OK, NOT_CONVERGED = 0, 1
EINVAL, ENOMEM, ESTATE, ECUDA, ENONFINITE, EDIVERGED, ETIMEOUT = -1, -2, -3, -4, -5, -6, -7
ESCRATCH = -8
NOALLOC_MAX_BLOCKS = 65536
STATUS_NAMES = {0: "OK", 1: "NOT_CONVERGED", -1: "EINVAL", -2: "ENOMEM", -3: "ESTATE",
                -4: "ECUDA", -5: "ENONFINITE", -6: "EDIVERGED", -7: "ETIMEOUT", -8: "ESCRATCH"}

_ALLOC = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
_FREE = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class hlbm_options(C.Structure):
    _fields_ = [
        ("storage", C.c_int),
        ("u_in", C.c_double),
        ("u_solid", C.c_double * 3),
        ("tau_adj", C.c_double),
        ("objectives", C.c_int),
        ("ffa_x", C.c_int),
        ("ffa_y0", C.c_int), ("ffa_y1", C.c_int),
        ("ffa_z0", C.c_int), ("ffa_z1", C.c_int),
        ("diss_box", C.c_int * 6),
        ("design_box", C.c_int * 6),
        ("accum_stride", C.c_int),
        ("check_every", C.c_int),
        ("average_full_f", C.c_int),
        ("block_x", C.c_int),
        ("adjoint_solver", C.c_int),
        ("gmres_restart", C.c_int),
        ("gmres_inner", C.c_int),
        ("stream", C.c_void_p),
        ("dev_alloc", _ALLOC),
        ("dev_free", _FREE),
        ("alloc_user", C.c_void_p),
        ("collision", C.c_int),
        ("inflow_ux", C.c_void_p),
        ("adjoint_warm_start", C.c_int),
    ]


class hlbm_stats(C.Structure):
    _fields_ = [
        ("primal_steps", C.c_long),
        ("adjoint_iters", C.c_long),
        ("primal_ms", C.c_double),
        ("adjoint_ms", C.c_double),
        ("primal_launches", C.c_long),
        ("adjoint_launches", C.c_long),
        ("primal_bytes_per_lup_plain", C.c_double),
        ("adjoint_bytes_per_lup", C.c_double),
        ("kernels_total", C.c_long),
    ]


class HlbmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build it with `python paper_2606_31707_b300/build.py`")
    lib = C.CDLL(LIB_PATH)
    P = C.c_void_p
    sig = {
        "hlbm_velocity_set": (C.c_int, [C.c_int, P, P]),
        "hlbm_default_options": (None, [C.POINTER(hlbm_options), C.POINTER(C.c_int)]),
        "hlbm_create": (C.c_int, [C.POINTER(P), C.c_int, C.POINTER(C.c_int), C.c_double,
                                  C.c_double, C.POINTER(hlbm_options)]),
        "hlbm_set_porosity": (C.c_int, [P, P, C.c_int, C.c_int]),
        "hlbm_configure": (C.c_int, [P, C.c_double, C.c_double, C.POINTER(hlbm_options)]),
        "hlbm_init_equilibrium": (C.c_int, [P, P, P, C.c_int, C.c_int]),
        "hlbm_run_primal": (C.c_int, [P, C.c_long, C.c_long]),
        "hlbm_run_tangent": (C.c_int, [P, C.c_long, P, C.c_int, C.c_int, C.c_int, P]),
        "hlbm_objective": (C.c_int, [P, C.c_int, C.POINTER(C.c_double)]),
        "hlbm_solve_adjoint": (C.c_int, [P, C.c_int, C.c_int, C.c_double, C.c_long,
                                         C.POINTER(C.c_long), C.POINTER(C.c_double)]),
        "hlbm_gradient": (C.c_int, [P, P, C.c_int, C.c_int]),
        "hlbm_get_field": (C.c_int, [P, C.c_int, P, C.c_int, C.c_int]),
        "hlbm_set_field": (C.c_int, [P, C.c_int, P, C.c_int, C.c_int]),
        "hlbm_get_stats": (C.c_int, [P, C.POINTER(hlbm_stats)]),
        "hlbm_save": (C.c_int, [P, C.c_char_p]),
        "hlbm_load": (C.c_int, [P, C.c_char_p]),
        "hlbm_last_error": (C.c_char_p, [P]),
        "hlbm_destroy": (None, [P]),
        "hlbm_batch_create": (C.c_int, [C.POINTER(P), C.c_int, P]),
        "hlbm_batch_run_primal": (C.c_int, [P, C.POINTER(P), C.c_int, C.c_long, C.c_long]),
        "hlbm_batch_solve_adjoint": (C.c_int, [P, C.POINTER(P), C.c_int, C.POINTER(C.c_int), C.c_int,
                                               C.c_double, C.c_long, C.POINTER(C.c_long),
                                               C.POINTER(C.c_double), C.POINTER(C.c_int)]),
        "hlbm_batch_destroy": (None, [P]),
        "hlbm_objective_noalloc": (C.c_int, [C.c_int, C.POINTER(C.c_int), C.c_double, C.c_double,
                                             C.c_double, C.POINTER(C.c_double), C.c_int,
                                             C.POINTER(C.c_int), P, P, P, P, P, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()
EXPORTED = ("hlbm_velocity_set", "hlbm_default_options", "hlbm_create", "hlbm_configure",
            "hlbm_set_porosity",
            "hlbm_init_equilibrium", "hlbm_run_primal", "hlbm_run_tangent", "hlbm_objective", "hlbm_solve_adjoint",
            "hlbm_gradient", "hlbm_get_field", "hlbm_set_field", "hlbm_get_stats", "hlbm_save",
            "hlbm_load", "hlbm_last_error", "hlbm_destroy", "hlbm_batch_create",
            "hlbm_batch_run_primal", "hlbm_batch_solve_adjoint", "hlbm_batch_destroy",
            "hlbm_objective_noalloc")


def lib():
    return _lib


# ---------------------------------------------------------------------------
# buffer marshalling
# ---------------------------------------------------------------------------

def _buf(x, writable=False):
    """(pointer, dtype code, on_device, keepalive) of a numpy array or torch tensor."""
    try:
        import torch
        if isinstance(x, torch.Tensor):
            if not x.is_contiguous():
                raise ValueError("tensor must be contiguous")
            if x.dtype == torch.float64:
                dt = DTYPE_F64
            elif x.dtype == torch.float32:
                dt = DTYPE_F32
            else:
                raise ValueError("float32 or float64 required")
            return C.c_void_p(x.data_ptr()), dt, int(x.is_cuda), x
    except ImportError:
        pass
    a = np.asarray(x)
    if a.dtype == np.float64:
        dt = DTYPE_F64
    elif a.dtype == np.float32:
        dt = DTYPE_F32
    else:
        a = a.astype(np.float64)
        dt = DTYPE_F64
    if writable:
        if not a.flags["C_CONTIGUOUS"] or not a.flags["WRITEABLE"]:
            raise ValueError("output array must be C-contiguous and writable")
    else:
        a = np.ascontiguousarray(a)
    return C.c_void_p(a.ctypes.data), dt, 0, a


def _check(ctx, status):
    if status < 0:
        msg = _lib.hlbm_last_error(ctx)
        raise HlbmError(status, msg.decode() if msg else "")
    return status


# ---------------------------------------------------------------------------
# the C entry points, same names
# ---------------------------------------------------------------------------

def hlbm_velocity_set(lattice: int):
    q = lattice
    xi = (C.c_int * (3 * q))()
    w = (C.c_double * q)()
    r = _lib.hlbm_velocity_set(lattice, xi, w)
    if r < 0:
        raise HlbmError(r, "bad lattice")
    return np.array(xi, dtype=np.int64).reshape(q, 3), np.array(w)


def hlbm_default_options(dims: Sequence[int]) -> hlbm_options:
    o = hlbm_options()
    d = (C.c_int * 3)(*dims)
    _lib.hlbm_default_options(C.byref(o), d)
    return o


def hlbm_create(lattice: int, dims: Sequence[int], tau: float, Cs: float,
                opt: Optional[hlbm_options] = None):
    ctx = C.c_void_p()
    d = (C.c_int * 3)(*dims)
    r = _lib.hlbm_create(C.byref(ctx), lattice, d, tau, Cs, C.byref(opt) if opt is not None else None)
    if r < 0:
        raise HlbmError(r, "hlbm_create failed")
    return ctx


def hlbm_configure(ctx, tau: float, Cs: float, opt: Optional[hlbm_options] = None):
    return _check(ctx, _lib.hlbm_configure(ctx, tau, Cs, C.byref(opt) if opt is not None else None))


def hlbm_set_porosity(ctx, d):
    p, dt, dev, keep = _buf(d)
    return _check(ctx, _lib.hlbm_set_porosity(ctx, p, dt, dev))


def hlbm_init_equilibrium(ctx, rho=None, u=None):
    dt, dev = DTYPE_F64, 0
    pr = pu = None
    keep = []
    if rho is not None:
        pr, dt, dev, k = _buf(rho)
        keep.append(k)
    if u is not None:
        pu, dtu, devu, k = _buf(u)
        keep.append(k)
        if rho is not None and (dtu != dt or devu != dev):
            raise ValueError("rho and u must share dtype and device")
        dt, dev = dtu, devu
    return _check(ctx, _lib.hlbm_init_equilibrium(ctx, pr, pu, dt, dev))


def hlbm_run_primal(ctx, steps: int, avg_window: int):
    return _check(ctx, _lib.hlbm_run_primal(ctx, steps, avg_window))


def hlbm_run_tangent(ctx, steps: int, delta, objective: int) -> np.ndarray:
    p, dt, dev, keep = _buf(delta)
    out = np.empty(steps, dtype=np.float64)
    _check(ctx, _lib.hlbm_run_tangent(ctx, steps, p, dt, dev, objective,
                                      C.c_void_p(out.ctypes.data)))
    return out


def hlbm_objective(ctx, objective: int) -> float:
    J = C.c_double()
    _check(ctx, _lib.hlbm_objective(ctx, objective, C.byref(J)))
    return J.value


def hlbm_solve_adjoint(ctx, objective: int, mode: int, tol: float, max_iter: int):
    it = C.c_long()
    res = C.c_double()
    st = _check(ctx, _lib.hlbm_solve_adjoint(ctx, objective, mode, tol, max_iter,
                                              C.byref(it), C.byref(res)))
    return st, it.value, res.value


def hlbm_gradient(ctx, out):
    p, dt, dev, keep = _buf(out, writable=True)
    return _check(ctx, _lib.hlbm_gradient(ctx, p, dt, dev))


def hlbm_get_field(ctx, which: int, out):
    p, dt, dev, keep = _buf(out, writable=True)
    return _check(ctx, _lib.hlbm_get_field(ctx, which, p, dt, dev))


def hlbm_set_field(ctx, which: int, data):
    p, dt, dev, keep = _buf(data)
    return _check(ctx, _lib.hlbm_set_field(ctx, which, p, dt, dev))


def hlbm_get_stats(ctx) -> hlbm_stats:
    s = hlbm_stats()
    _check(ctx, _lib.hlbm_get_stats(ctx, C.byref(s)))
    return s


def hlbm_save(ctx, path: str):
    return _check(ctx, _lib.hlbm_save(ctx, path.encode()))


def hlbm_load(ctx, path: str):
    return _check(ctx, _lib.hlbm_load(ctx, path.encode()))


def hlbm_last_error(ctx) -> str:
    m = _lib.hlbm_last_error(ctx)
    return m.decode() if m else ""


def hlbm_destroy(ctx):
    _lib.hlbm_destroy(ctx)


def _ctx_array(ctxs):
    arr = (C.c_void_p * len(ctxs))()
    for k, c in enumerate(ctxs):
        arr[k] = c.value if isinstance(c, C.c_void_p) else c
    return arr


def _check_many(ctxs, status):
    if status < 0:
        for c in ctxs:
            m = _lib.hlbm_last_error(c)
            if m:
                raise HlbmError(status, m.decode())
        raise HlbmError(status, "batched call failed")
    return status


def hlbm_batch_create(lattice: int, stream: int):
    """A batch for contexts of this lattice created on ``stream`` (a cudaStream_t)."""
    b = C.c_void_p()
    r = _lib.hlbm_batch_create(C.byref(b), lattice, C.c_void_p(stream))
    if r < 0:
        raise HlbmError(r, "hlbm_batch_create failed")
    return b


def hlbm_batch_run_primal(batch, ctxs, steps: int, avg_window: int):
    return _check_many(ctxs, _lib.hlbm_batch_run_primal(batch, _ctx_array(ctxs), len(ctxs),
                                                        steps, avg_window))


def hlbm_batch_solve_adjoint(batch, ctxs, objectives, mode: int, tol: float, max_iter: int):
    """Returns (worst status, [(status, iterations, residual)] per context)."""
    n = len(ctxs)
    objs = (C.c_int * n)(*objectives)
    it = (C.c_long * n)()
    res = (C.c_double * n)()
    st = (C.c_int * n)()
    r = _lib.hlbm_batch_solve_adjoint(batch, _ctx_array(ctxs), n, objs, mode, tol, max_iter,
                                      it, res, st)
    if r < 0 and all(v >= 0 for v in st):
        _check_many(ctxs, r)
    return r, [(st[k], it[k], res[k]) for k in range(n)]


def hlbm_batch_destroy(batch):
    _lib.hlbm_batch_destroy(batch)


def hlbm_objective_noalloc(lattice: int, dims: Sequence[int], tau: float, Cs: float, u_in: float,
                           objective: int, region: Sequence[int], f, d, J, dJdf=None, dJdd=None,
                           stream: Optional[int] = None, u_solid=(0.0, 0.0, 0.0)) -> int:
    """Objective of a device-resident state without any allocation in the
    library (see include/hlbm.h).  f (q*N), d (N), J (1), dJdf (q*N) and dJdd
    (N) are contiguous float64 CUDA tensors on the current device; the C side
    cannot check their sizes, so they are checked here and a mismatch raises
    ValueError before anything is launched.  ``stream`` defaults to torch's
    current stream.  Returns the status (negative on error) without raising."""
    import torch

    q = int(lattice)
    if q not in (9, 19) or len(dims) != 3 or len(region) != 6:
        raise ValueError("lattice must be 9 or 19, dims 3 values, region 6 values")
    N = int(dims[0]) * int(dims[1]) * int(dims[2])
    dev = None
    sizes = {"f": q * N, "d": N, "J": 1, "dJdf": q * N, "dJdd": N}
    tensors = {"f": f, "d": d, "J": J, "dJdf": dJdf, "dJdd": dJdd}
    for name in ("f", "d", "J"):
        if tensors[name] is None:
            raise ValueError(f"{name} is required")
    for name, t in tensors.items():
        if t is None:
            continue
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")
        if t.dtype != torch.float64:
            raise ValueError(f"{name} must be float64")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        if dev is None:
            dev = torch.cuda.current_device()
        if t.device.index != dev:
            raise ValueError(f"{name} is on cuda:{t.device.index}, the current device is cuda:{dev}")
        if t.numel() != sizes[name]:
            raise ValueError(f"{name} needs {sizes[name]} elements, got {t.numel()}")
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    ptr = [C.c_void_p(t.data_ptr()) if t is not None else None for t in (f, d, J, dJdf, dJdd)]
    return _lib.hlbm_objective_noalloc(lattice, (C.c_int * 3)(*dims), tau, Cs, u_in,
                                       (C.c_double * 3)(*u_solid), objective,
                                       (C.c_int * 6)(*region), *ptr, C.c_void_p(stream))
