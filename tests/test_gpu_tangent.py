"""Tangent-linear primal (forward sensitivity along the trajectory, the
quantity the paper's App. C follows) against the oracle's step Jacobians and
against central differences of J along the porosity direction."""
import numpy as np
import pytest

from oracle import adjoint as oadj
from oracle import hlbm as ohlbm
from oracle import objectives as oobj
from tests.hlbm_cases import direction_perm, rel_l2
from workloads import Regions, cylinder_porosity

pytestmark = pytest.mark.gpu

H = pytest.importorskip("paper_2606_31707_b300.hlbm")
from paper_2606_31707_b300 import Solver  # noqa: E402


def _case(q, Cs):
    dims = (150, 16, 1) if q == 9 else (80, 10, 6)
    P = ohlbm.Params(q, dims, tau0=0.7, Cs=Cs, u_in=0.05)
    nx, ny, nz = dims
    d = cylinder_porosity(dims, 20.0, ny / 2.0, 3.0, 1.5, jitter=0.01, seed=2)
    R = Regions(ffa_x=nx - 30, ffa_y=(0, ny), ffa_z=(0, nz), diss_box=(2, nx - 10, 0, ny, 0, nz),
                design_box=(0, nx, 0, ny, 0, nz))
    rng = np.random.default_rng(4)
    delta = np.zeros(P.shape)
    delta[..., 15:26] = rng.standard_normal(delta[..., 15:26].shape)
    return P, d, R, delta


def _oracle_tangent(P, d, R, delta, steps, objective):
    f = ohlbm.initial_state(P)
    v = np.zeros_like(f)
    jd = []
    for _ in range(steps):
        g, gd = oobj.partials(f, d, P, objective, R)
        jd.append(float((g * v).sum() + (gd * delta).sum()))
        lin = oadj.Linearisation(f, d, P, oadj.EXACT, outlet="streamed")
        v = lin.jvp(v) + (lin.D @ delta.ravel()).reshape(f.shape)
        f = ohlbm.step(f, d, P)
    return np.array(jd)


@pytest.mark.parametrize("q,Cs", [(9, 0.0), (9, 0.15), (19, 0.1)])
@pytest.mark.parametrize("objective", [oobj.FFA, oobj.DISS])
def test_tangent_matches_oracle_step_jacobians(q, Cs, objective):
    P, d, R, delta = _case(q, Cs)
    steps = 25
    s = Solver(q, P.dims, P.tau0, P.Cs, storage=H.FP64, u_in=P.u_in, regions=R)
    s.set_porosity(d)
    got = H.hlbm_run_tangent(s.ctx, steps, np.ascontiguousarray(delta.ravel()), objective)
    s.close()
    ref = _oracle_tangent(P, d, R, delta, steps, objective)
    assert rel_l2(got[1:], ref[1:]) <= 1e-10


def test_tangent_matches_central_differences_of_the_objective():
    P, d, R, delta = _case(9, 0.0)
    steps, h = 40, 1e-6
    s = Solver(9, P.dims, P.tau0, 0.0, storage=H.FP64, u_in=P.u_in, regions=R)
    s.set_porosity(d)
    got = H.hlbm_run_tangent(s.ctx, steps, np.ascontiguousarray(delta.ravel()), oobj.DISS)
    s.close()
    Js = []
    for sgn in (1, -1):
        f = ohlbm.initial_state(P)
        dd = d + sgn * h * delta
        hist = []
        for _ in range(steps):
            hist.append(oobj.value(f, dd, P, oobj.DISS, R))
            f = ohlbm.step(f, dd, P)
        Js.append(np.array(hist))
    fd = (Js[0] - Js[1]) / (2 * h)
    assert rel_l2(got[1:], fd[1:]) <= 1e-6


@pytest.mark.parametrize("q,Cs", [(9, 0.0), (9, 0.15), (19, 0.1)])
def test_tangent_mean_matches_the_unsteady_adjoint_reference(q, Cs):
    # d J_T / dd . delta for the short-horizon average J_T = (1/T) sum_n J(f^n):
    # the mean of the GPU tangent's per-step derivatives against the oracle's
    # checkpointed unsteady adjoint (duality of forward and reverse mode)
    P, d, R, delta = _case(q, Cs)
    T = 30
    s = Solver(q, P.dims, P.tau0, P.Cs, storage=H.FP64, u_in=P.u_in, regions=R)
    s.set_porosity(d)
    jd = H.hlbm_run_tangent(s.ctx, T, np.ascontiguousarray(delta.ravel()), oobj.DISS)
    s.close()
    G, _, _ = oadj.unsteady_adjoint_gradient(ohlbm.initial_state(P), d, P, T, oobj.DISS, R)
    ref = float((G * delta).sum())
    assert abs(float(np.mean(jd)) - ref) <= 1e-10 * max(abs(ref), 1e-12)
