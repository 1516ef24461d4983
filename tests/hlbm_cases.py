"""Shared helpers of the tests: oracle runs of a workload and the mapping
between the library's direction order and the oracle's.

Test infrastructure only (it imports the oracle)."""
from __future__ import annotations

import numpy as np

from oracle import adjoint as oadj
from oracle import hlbm as ohlbm
from oracle import meanflow as omf
from oracle import objectives as oobj
from oracle.hlbm import Params


def direction_perm(lib_xi: np.ndarray, P: Params) -> np.ndarray:
    """perm[k] = oracle index of the library's direction k (same xi)."""
    perm = []
    for v in lib_xi:
        hit = np.nonzero((P.xi == v).all(axis=1))[0]
        assert hit.size == 1
        perm.append(int(hit[0]))
    return np.array(perm)


def to_lib(field_oracle: np.ndarray, perm) -> np.ndarray:
    return np.ascontiguousarray(field_oracle[perm])


def rel_l2(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.sqrt((b * b).sum())
    return float(np.sqrt(((a - b) ** 2).sum()) / (den if den > 0 else 1.0))


def params_of(wl, tau=None, Cs=None):
    tau0 = ohlbm.tau_from_reynolds(wl.u0, wl.L, wl.Re) if tau is None else tau
    return Params(wl.q, wl.dims, tau0=tau0, Cs=wl.Cs if Cs is None else Cs, u_in=wl.u0)


def oracle_pipeline(P, d, regions, f0, steps, W, objective, mode=oadj.EXACT, tau_adj=None,
                    stride=1, direct=True, tol=1e-13, mask=3):
    """Primal with averages, adjoint and gradient, all in the oracle."""
    out = omf.run_primal(f0, d, P, steps, W, regions, mask, stride)
    lin = oadj.Linearisation(out["fbar"], d, P, mode, tau_adj, out["tau_t_bar"])
    g = out[("gbar", objective)]
    if direct:
        lam = oadj.solve_adjoint_direct(lin, g)
    else:
        lam, _, _ = oadj.solve_adjoint(lin, g, tol=tol, max_iter=1_000_000)
    G = oadj.gradient(lin, lam, out[("dJdd_bar", objective)])
    return dict(out=out, lin=lin, lam=lam, G=G, mu=lin.mu(lam))


def oracle_grf_gradients():
    """The Gaussian-random-field design case (D2Q9 400x160, Re 40) in the
    oracle: steady state by Newton steps with the exact step Jacobian, the
    steady adjoint by a sparse direct solve, and the gradient and J of both
    objectives (Eq. gradients_steady).  Returns {"newton_residual": r,
    1: (G, J) of J_FFA, 2: (G, J) of J_DISS}.  Picklable for a spawned worker."""
    from workloads import make_workload

    wl = make_workload("grf2d_re40")
    P = Params(9, wl.dims, tau0=ohlbm.tau_from_reynolds(wl.u0, wl.L, wl.Re), u_in=wl.u0)
    d = wl.porosity
    f = ohlbm.initial_state(P)
    for _ in range(1000):
        f = ohlbm.step(f, d, P)
    f, res = oadj.newton_steady(f, d, P, iters=20, tol=1e-12)
    lin = oadj.Linearisation(f, d, P, oadj.EXACT)
    out = {"newton_residual": res}
    for o in (oobj.FFA, oobj.DISS):
        g, gd = oobj.partials(f, d, P, o, wl.regions)
        lam = oadj.solve_adjoint_direct(lin, g)
        out[o] = (oadj.gradient(lin, lam, gd), oobj.value(f, d, P, o, wl.regions))
    return out
