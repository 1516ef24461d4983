"""Primal run with tracking averages (Sec. 3.3, Eq. averageObjective; Sec. 5.3
and 5.4 for the averaging windows).

Readings:
* ``steps`` time steps are taken from the given canonical state.  The last
  ``avg_window`` of them sample the canonical state they start from, every
  ``stride``-th one; the averages divide by the number of samples taken
  (the paper's 1/(t_e - t_s) normaliser read as 1/#samples).
* Averaged entities (Sec. 3.3 and App. A): the populations f (their mean is
  the linearisation point of the mean-flow adjoint), J, dJ/df, dJ/dd, and
  the turbulent part tau_eff - tau0 of the relaxation time (used by the
  frozen-turbulence assumption, Sec. 5.4).
* avg_window = 1 is the steady case: f_bar is the last state sampled.
"""
from __future__ import annotations

import numpy as np

from . import objectives as obj
from .hlbm import Params, local_state, step


def run_primal(f, d, P: Params, steps: int, avg_window: int, regions=None,
               objective_mask: int = obj.FFA | obj.DISS, stride: int = 1):
    """Advance ``steps`` steps; average the last ``avg_window`` canonical states."""
    if avg_window > steps or avg_window < 1:
        raise ValueError("need 1 <= avg_window <= steps")
    first = steps - avg_window
    acc = dict(fsum=np.zeros_like(f), tsum=np.zeros(f.shape[1:]), n=0)
    objs = [o for o in (obj.FFA, obj.DISS, obj.MEA) if objective_mask & o] if regions is not None else []
    for o in objs:
        acc[("g", o)] = np.zeros_like(f)
        acc[("dd", o)] = np.zeros(f.shape[1:])
        acc[("J", o)] = 0.0
    for n in range(steps):
        if n >= first and (n - first) % stride == 0:
            acc["fsum"] += f
            acc["tsum"] += local_state(f, d, P)["tau"] - P.tau0
            for o in objs:
                g, dd = obj.partials(f, d, P, o, regions)
                acc[("g", o)] += g
                acc[("dd", o)] += dd
                acc[("J", o)] += obj.value(f, d, P, o, regions)
            acc["n"] += 1
        f = step(f, d, P)
    n = acc["n"]
    out = dict(f=f, fbar=acc["fsum"] / n, tau_t_bar=acc["tsum"] / n, nsamples=n)
    for o in objs:
        out[("gbar", o)] = acc[("g", o)] / n
        out[("dJdd_bar", o)] = acc[("dd", o)] / n
        out[("Jbar", o)] = acc[("J", o)] / n
    return out
