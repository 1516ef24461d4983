"""Parity of the LES configuration at quarter scale (D3Q19 160x80x25, the
cylinder of diameter 8 at (40, 40), Smagorinsky C_S = 0.1, tau0 from Re 3900
at u0 = 0.05, BGK collision) against the FP64 oracle.

From the same canonical state both sides run a short primal with a tracking
window; the GPU's own averages are compared with the oracle's, then each side
linearises at its own averaged state and runs the same number of adjoint
sweeps from zero (a well-defined value whether or not the fixed point
contracts) and contracts the gradient.  Covered: the exact LES linearisation
and the frozen-turbulence one (Sec. 5.4), each with tau_adj in {tau0, 0.6,
0.65} (the adjoint regularisation of Sec. 5.4), FP32 populations (bound
1e-4 on the gradient) and FP16 deviation storage (stated bound below).

The oracle keeps the collision Jacobian as per-cell blocks here
(``Linearisation(..., assemble=False)``): the assembled 19 x 19 x 320 000
matrices would not fit a test's memory budget."""
import numpy as np
import pytest

from oracle import adjoint as oadj
from oracle import hlbm as ohlbm
from oracle import meanflow as omf
from oracle import objectives as oobj
from tests.hlbm_cases import direction_perm, rel_l2, to_lib
from workloads import make_workload

pytestmark = pytest.mark.gpu

H = pytest.importorskip("paper_2606_31707_b300.hlbm")
from paper_2606_31707_b300 import Solver  # noqa: E402

STEPS, WINDOW, SWEEPS = 4, 3, 10
TOL_FP32 = 1e-4      # gradient and mu, FP32 populations and arithmetic
TOL_FP32_AVG = 1e-5  # averaged fields (a few FP32 steps)
# FP16 deviation storage: each stored population carries a relative rounding
# of 2^-11 of its deviation from w_i; the averaged state and everything
# linearised about it inherit that, measured at 1.4e-3 (f_bar) and 5e-3 (G)
TOL_FP16_AVG = 5e-3
TOL_FP16 = 2e-2

MODES = [(oadj.EXACT, None), (oadj.EXACT, 0.6), (oadj.EXACT, 0.65),
         (oadj.FTA, None), (oadj.FTA, 0.6), (oadj.FTA, 0.65)]


def _initial_state(P, seed=12):
    # equilibrium of a seeded flow with 10 % velocity noise plus 1 % population
    # noise: every cell has a non-trivial stress, so the LES relaxation time and
    # its derivative are active everywhere, not only at the cylinder
    rng = np.random.default_rng(seed)
    u = np.zeros((3,) + P.shape)
    u[0] = P.u_in * (1 + 0.1 * rng.standard_normal(P.shape))
    u[1] = 0.1 * P.u_in * rng.standard_normal(P.shape)
    u[2] = 0.1 * P.u_in * rng.standard_normal(P.shape)
    f = ohlbm.equilibrium(np.ones(P.shape), u, P) * (1 + 0.01 * rng.standard_normal((P.q,) + P.shape))
    return ohlbm.apply_boundary(f, P)


@pytest.fixture(scope="module")
def case():
    wl = make_workload("les3d_re3900_quarter")
    P = ohlbm.Params(19, wl.dims, tau0=ohlbm.tau_from_reynolds(wl.u0, wl.L, wl.Re), Cs=wl.Cs,
                     u_in=wl.u0)
    f0 = _initial_state(P)
    out = omf.run_primal(f0, wl.porosity, P, STEPS, WINDOW, wl.regions, 3)
    refs = {}
    for mode, tadj in MODES:
        lin = oadj.Linearisation(out["fbar"], wl.porosity, P, mode, tadj, out["tau_t_bar"],
                                 assemble=False)
        objs = (oobj.FFA, oobj.DISS) if (mode, tadj) == (oadj.EXACT, 0.6) else (oobj.FFA,)
        for o in objs:
            lam, _, _ = oadj.solve_adjoint(lin, out[("gbar", o)], tol=0.0, max_iter=SWEEPS)
            refs[(mode, tadj, o)] = (lin.mu(lam), oadj.gradient(lin, lam, out[("dJdd_bar", o)]))
        del lin
    return wl, P, f0, out, refs


def _gpu_run(wl, P, f0, storage, tau_adj):
    s = Solver(19, wl.dims, P.tau0, P.Cs, storage=storage, u_in=wl.u0, regions=wl.regions,
               tau_adj=tau_adj or 0.0)
    perm = direction_perm(s.xi, P)
    s.set_porosity(wl.porosity)
    s.set_field(H.FIELD_F, to_lib(f0, perm))
    s.run_primal(STEPS, WINDOW)
    return s, perm


def _check_averages(s, perm, out, tol):
    assert rel_l2(s.field(H.FIELD_FBAR) - s.w[:, None, None, None],
                  to_lib(out["fbar"], perm) - s.w[:, None, None, None]) <= tol
    assert rel_l2(s.field(H.FIELD_TAU_T), out["tau_t_bar"]) <= tol
    for o, gf, df in ((oobj.FFA, H.FIELD_GBAR_FFA, H.FIELD_DJDD_FFA),
                      (oobj.DISS, H.FIELD_GBAR_DISS, H.FIELD_DJDD_DISS)):
        assert rel_l2(s.field(gf), to_lib(out[("gbar", o)], perm)) <= tol
        if o == oobj.DISS:
            assert rel_l2(s.field(df), out[("dJdd_bar", o)]) <= tol
        assert abs(s.objective(o) - out[("Jbar", o)]) <= tol * abs(out[("Jbar", o)])


def _check_adjoint(s, perm, refs, mode, tadj, objs, tol):
    errs = []
    for o in objs:
        st, it, res = s.solve_adjoint(o, mode, 0.0, SWEEPS)
        assert st == H.NOT_CONVERGED and it == SWEEPS  # a fixed sweep count, tol 0
        mu_ref, G_ref = refs[(mode, tadj, o)]
        e_mu = rel_l2(s.field(H.FIELD_LAMBDA), to_lib(mu_ref, perm))
        e_g = rel_l2(s.gradient(), G_ref)
        errs.append((o, e_mu, e_g))
        assert e_mu <= tol and e_g <= tol, (mode, tadj, o, e_mu, e_g)
    return errs


@pytest.mark.parametrize("mode,tadj", MODES)
def test_quarter_les_fp32_averages_adjoint_and_gradient(case, mode, tadj):
    wl, P, f0, out, refs = case
    s, perm = _gpu_run(wl, P, f0, H.FP32, tadj)
    _check_averages(s, perm, out, TOL_FP32_AVG)
    objs = (oobj.FFA, oobj.DISS) if (mode, tadj) == (oadj.EXACT, 0.6) else (oobj.FFA,)
    errs = _check_adjoint(s, perm, refs, mode, tadj, objs, TOL_FP32)
    print("quarter LES FP32", mode, tadj, errs)
    s.close()


def test_quarter_les_fp16_deviation_storage_within_its_stated_bound(case):
    wl, P, f0, out, refs = case
    s, perm = _gpu_run(wl, P, f0, H.FP16DEV, 0.6)
    _check_averages(s, perm, out, TOL_FP16_AVG)
    errs = _check_adjoint(s, perm, refs, oadj.EXACT, 0.6, (oobj.FFA, oobj.DISS), TOL_FP16)
    print("quarter LES FP16", errs)
    s.close()
