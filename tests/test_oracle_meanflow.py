"""Pins of the oracle's tracking averages (Sec. 3.3, Eq. averageObjective;
Sec. 5.4 for the averaged turbulent relaxation time of the frozen-turbulence
adjoint) against an explicit history of canonical states.

Every averaged field is recomputed here from the stored states by a route
that does not go through ``meanflow.run_primal``: the turbulent part of the
relaxation time by a fixed-point iteration of the Smagorinsky definition
(nu_t = C_S^2 |S|, S = -Pi / (2 tau_eff c_s^2), tau_eff = tau0 + nu_t / c_s^2,
Sec. 2.2) with Pi from the closed-form equilibrium second moment, and the
objective derivatives from ``objectives.partials`` (pinned by central
differences elsewhere).  The window and stride are chosen so that the
sample count (3) differs from the window length (5), so a wrong normaliser
fails too."""
import numpy as np
import pytest

from oracle import hlbm
from oracle import meanflow
from oracle import objectives as obj
from oracle.hlbm import Params
from workloads import Regions, cylinder_porosity

CS2 = 1.0 / 3.0


def _case(q, Cs):
    dims = (24, 12, 1) if q == 9 else (14, 8, 4)
    P = Params(q, dims, tau0=0.56, Cs=Cs, u_in=0.06)
    d = cylinder_porosity(dims, 7.0, dims[1] / 2.0, 2.0, 1.2, jitter=0.01, seed=5)
    nx, ny, nz = dims
    R = Regions(ffa_x=nx - 5, ffa_y=(0, ny), ffa_z=(0, nz),
                diss_box=(2, nx - 3, 0, ny, 0, nz), design_box=(0, nx, 0, ny, 0, nz))
    return P, d, R


def _tau_turb_by_fixed_point(f, d, P):
    """tau_eff - tau0 of the Smagorinsky model, from its definition.

    Pi = sum_i xi_i xi_i f_i - (rho c_s^2 I + rho u~ u~): the equilibrium's
    second moment in closed form.  tau_eff = tau0 + C_S^2 |S| / c_s^2 with
    |S| = sqrt(2 S:S), S = -Pi / (2 tau_eff c_s^2), solved by fixed-point
    iteration (a contraction: the right side changes by C_S^2 ... / tau^2)."""
    xi = P.xif
    rho = f.sum(axis=0)
    u = np.einsum("ia,i...->a...", xi, f) / rho
    ut = d * u  # solid velocity 0
    M2 = np.einsum("ia,ib,i...->ab...", xi, xi, f)
    I = np.diag([1.0, 1.0, 1.0 if P.q == 19 else 0.0])
    Pi = M2 - rho * CS2 * I.reshape(3, 3, *([1] * rho.ndim)) - rho * np.einsum("a...,b...->ab...", ut, ut)
    tau = np.full(rho.shape, P.tau0)
    for _ in range(200):
        S = -Pi / (2.0 * tau * CS2)
        Snorm = np.sqrt(2.0 * np.einsum("ab...,ab...->...", S, S))
        tau = P.tau0 + P.Cs ** 2 * Snorm / CS2
    return tau - P.tau0


@pytest.mark.parametrize("q,Cs", [(9, 0.2), (19, 0.15)])
def test_averaged_tau_turb_and_dJdd_match_history(q, Cs):
    P, d, R = _case(q, Cs)
    f = hlbm.initial_state(P)
    steps, W, stride = 14, 5, 2
    first = steps - W
    tts, dds, Js = [], {o: [] for o in (obj.FFA, obj.DISS)}, {o: [] for o in (obj.FFA, obj.DISS)}
    for n in range(steps):
        if n >= first and (n - first) % stride == 0:
            tts.append(_tau_turb_by_fixed_point(f, d, P))
            for o in (obj.FFA, obj.DISS):
                dds[o].append(obj.partials(f, d, P, o, R)[1])
                Js[o].append(obj.value(f, d, P, o, R))
        f = hlbm.step(f, d, P)
    assert len(tts) == 3
    out = meanflow.run_primal(hlbm.initial_state(P), d, P, steps, W, R, obj.FFA | obj.DISS,
                              stride=stride)
    assert out["nsamples"] == 3
    ref_t = np.mean(tts, axis=0)
    assert np.abs(ref_t).max() > 1e-4  # the turbulent part is not trivially zero here
    assert np.abs(out["tau_t_bar"] - ref_t).max() <= 1e-12 * np.abs(ref_t).max()
    for o in (obj.FFA, obj.DISS):
        ref_dd = np.mean(dds[o], axis=0)
        if o == obj.FFA:
            # J_FFA does not depend on d (Sec. 4.2)
            assert np.abs(out[("dJdd_bar", o)]).max() == 0.0
            continue
        assert np.abs(ref_dd).max() > 0
        assert np.abs(out[("dJdd_bar", o)] - ref_dd).max() <= 1e-14 * np.abs(ref_dd).max()
    for o in (obj.FFA, obj.DISS):
        assert abs(out[("Jbar", o)] - np.mean(Js[o])) <= 1e-14 * abs(np.mean(Js[o]))


def test_tau_turb_average_is_zero_without_les():
    P, d, R = _case(9, 0.0)
    out = meanflow.run_primal(hlbm.initial_state(P), d, P, 6, 3, R)
    assert np.abs(out["tau_t_bar"]).max() == 0.0
