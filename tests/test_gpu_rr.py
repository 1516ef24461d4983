"""Parity of the recursive regularised collision (Sec. 2.2, Eq. HRRLBM) on
the CUDA path with the FP64 oracle: primal steps, the averages of a window,
and the mean-flow adjoint and gradient (exact and frozen turbulence,
D2Q9 and D3Q19).  The library linearises from its averaged moments up to
second order; the oracle linearises at the averaged populations."""
import functools
import os
import tempfile

import numpy as np
import pytest

from oracle import adjoint as oadj
from oracle import hlbm as ohlbm
from oracle import meanflow as omf
from oracle import objectives as oobj
from tests.hlbm_cases import direction_perm, rel_l2, to_lib
from workloads import Regions, cylinder_porosity

pytestmark = pytest.mark.gpu

H = pytest.importorskip("paper_2606_31707_b300.hlbm")
from paper_2606_31707_b300 import Solver  # noqa: E402


def _case(q=9, dims=(300, 24, 1), Cs=0.0, tau=0.7, u_in=0.05, seed=0):
    P = ohlbm.Params(q, dims, tau0=tau, Cs=Cs, u_in=u_in, collision="rr")
    nx, ny, nz = dims
    d = cylinder_porosity(dims, 30.0, ny / 2.0, 4.0, 1.5, jitter=0.01, seed=seed)
    regions = Regions(ffa_x=nx // 2 + 7, ffa_y=(0, ny), ffa_z=(0, nz),
                      diss_box=(3, nx - 37, 1, ny - 2, 0, nz),
                      design_box=(5, nx - 3, 0, ny, 0, nz))
    return P, d, regions


def _solver(P, R, storage, **kw):
    return Solver(P.q, P.dims, P.tau0, P.Cs, storage=storage, u_in=P.u_in, regions=R,
                  collision=H.COLL_RR, **kw)


def _perturbed_state(P, seed=1, amp=0.01):
    rng = np.random.default_rng(seed)
    u = np.zeros((3,) + P.shape)
    u[0] = P.u_in * (1 + 0.2 * rng.standard_normal(P.shape))
    u[1] = 0.01 * rng.standard_normal(P.shape)
    if P.q == 19:
        u[2] = 0.01 * rng.standard_normal(P.shape)
    rho = 1 + 0.01 * rng.standard_normal(P.shape)
    f = ohlbm.equilibrium(rho, u, P) * (1 + amp * rng.standard_normal((P.q,) + P.shape))
    return ohlbm.apply_boundary(f, P)


@pytest.mark.parametrize("q,dims,Cs,storage,tol", [
    (9, (300, 24, 1), 0.0, H.FP64, 1e-13),
    (9, (300, 24, 1), 0.2, H.FP64, 1e-13),
    (19, (150, 10, 6), 0.15, H.FP64, 1e-13),
    (9, (300, 24, 1), 0.0, H.FP32, 1e-6),
    (19, (150, 10, 6), 0.15, H.FP32, 1e-6),
])
@pytest.mark.parametrize("steps", [1, 2, 7])
def test_rr_primal_steps_match_oracle(q, dims, Cs, storage, tol, steps):
    P, d, R = _case(q, dims, Cs)
    f0 = _perturbed_state(P)
    s = _solver(P, R, storage)
    perm = direction_perm(s.xi, P)
    s.set_porosity(d)
    s.set_field(H.FIELD_F, to_lib(f0, perm))
    s.run_primal(steps, 0)
    f = f0
    for _ in range(steps):
        f = ohlbm.step(f, d, P)
    assert rel_l2(s.field(H.FIELD_F), to_lib(f, perm)) <= tol
    s.close()


def test_rr_differs_from_bgk_on_the_device():
    # the collision option reaches the kernels
    P, d, R = _case(9, (300, 24, 1), 0.0)
    f0 = _perturbed_state(P)
    out = []
    for coll in (H.COLL_BGK, H.COLL_RR):
        s = Solver(P.q, P.dims, P.tau0, 0.0, storage=H.FP64, u_in=P.u_in, regions=R, collision=coll)
        perm = direction_perm(s.xi, P)
        s.set_porosity(d)
        s.set_field(H.FIELD_F, to_lib(f0, perm))
        s.run_primal(3, 0)
        out.append(s.field(H.FIELD_F))
        s.close()
    assert rel_l2(out[0], out[1]) > 1e-6


@pytest.mark.parametrize("storage,tol", [(H.FP16DEV, 3e-3), (H.BF16DEV, 3e-2)])
def test_rr_16bit_deviation_storage_bound(storage, tol):
    P, d, R = _case(9, (300, 24, 1), 0.0)
    f0 = _perturbed_state(P, amp=0.0)
    s = _solver(P, R, storage)
    perm = direction_perm(s.xi, P)
    s.set_porosity(d)
    s.set_field(H.FIELD_F, to_lib(f0, perm))
    s.run_primal(20, 0)
    f = f0
    for _ in range(20):
        f = ohlbm.step(f, d, P)
    dev_ref = to_lib(f, perm) - s.w[:, None, None, None]
    assert rel_l2(s.field(H.FIELD_F) - s.w[:, None, None, None], dev_ref) <= tol
    s.close()


@pytest.mark.parametrize("q,dims,Cs", [(9, (300, 24, 1), 0.0), (9, (300, 24, 1), 0.2),
                                      (19, (150, 10, 6), 0.15)])
def test_rr_averages_match_oracle(q, dims, Cs):
    P, d, R = _case(q, dims, Cs)
    f0 = _perturbed_state(P)
    s = _solver(P, R, H.FP64, accum_stride=2, average_full_f=True)
    perm = direction_perm(s.xi, P)
    s.set_porosity(d)
    s.set_field(H.FIELD_F, to_lib(f0, perm))
    s.run_primal(12, 7)
    out = omf.run_primal(f0, d, P, 12, 7, R, 3, stride=2)
    assert rel_l2(s.field(H.FIELD_FBAR), to_lib(out["fbar"], perm)) <= 1e-13
    for o, gf in ((oobj.FFA, H.FIELD_GBAR_FFA), (oobj.DISS, H.FIELD_GBAR_DISS)):
        assert rel_l2(s.field(gf), to_lib(out[("gbar", o)], perm)) <= 1e-11
        assert abs(s.objective(o) - out[("Jbar", o)]) <= 1e-12 * max(1.0, abs(out[("Jbar", o)]))
    if Cs > 0:
        assert rel_l2(s.field(H.FIELD_TAU_T), out["tau_t_bar"]) <= 1e-11
    s.close()


@functools.lru_cache(maxsize=None)
def _settled(q, dims, Cs, steps):
    """The state the oracle reaches after `steps` regularised steps of the
    window cases' flow (tau 0.8, u_in 0.04) from rest.  Cached: several tests
    share a case."""
    P, d, _ = _case(q, dims, Cs, tau=0.8, u_in=0.04)
    f = ohlbm.initial_state(P)
    for _ in range(steps):
        f = ohlbm.step(f, d, P)
    f.setflags(write=False)
    return f


def _window_gpu_vs_oracle(q, dims, Cs, storage, objective, mode, tau_adj=None, settle=2950, W=50):
    """Mean-flow adjoint over a window of W steps from a state the oracle
    reached after `settle` steps (written into the library): both sides
    average the same window from the same state."""
    P, d, R = _case(q, dims, Cs, tau=0.8, u_in=0.04)
    s = _solver(P, R, storage, tau_adj=tau_adj or 0.0)
    perm = direction_perm(s.xi, P)
    s.set_porosity(d)
    f_start = _settled(q, dims, Cs, settle)
    s.set_field(H.FIELD_F, to_lib(f_start, perm))
    s.run_primal(W, W)
    out = omf.run_primal(f_start, d, P, W, W, R, 3)
    lin = oadj.Linearisation(out["fbar"], d, P, mode, tau_adj, out["tau_t_bar"])
    lam = oadj.solve_adjoint_direct(lin, out[("gbar", objective)])
    G = oadj.gradient(lin, lam, out[("dJdd_bar", objective)])
    st, it, res = s.solve_adjoint(objective, mode, 1e-13 if storage == H.FP64 else 1e-7, 400000)
    Gg = s.gradient()
    mu = s.field(H.FIELD_LAMBDA)
    s.close()
    b = R.design_box
    return Gg, G[b[4]:b[5], b[2]:b[3], b[0]:b[1]], mu, to_lib(lin.mu(lam), perm), st


@pytest.mark.parametrize("objective", [oobj.FFA, oobj.DISS])
@pytest.mark.parametrize("q,dims,Cs,mode", [
    (9, (300, 24, 1), 0.0, oadj.EXACT),
    (9, (300, 24, 1), 0.15, oadj.EXACT),
    (9, (300, 24, 1), 0.15, oadj.FTA),
    (19, (140, 10, 4), 0.1, oadj.EXACT),
    (19, (140, 10, 4), 0.1, oadj.FTA),
])
def test_rr_mean_flow_gradient_fp64_matches_oracle(q, dims, Cs, mode, objective):
    Gg, Gref, mu, mu_ref, st = _window_gpu_vs_oracle(q, dims, Cs, H.FP64, objective, mode)
    assert st == H.OK
    assert rel_l2(Gg, Gref) <= 1e-9
    assert rel_l2(mu, mu_ref) <= 1e-9


def test_rr_gradient_fp32_matches_oracle():
    Gg, Gref, _, _, st = _window_gpu_vs_oracle(9, (300, 24, 1), 0.0, H.FP32, oobj.DISS, oadj.EXACT)
    assert st in (H.OK, H.NOT_CONVERGED)
    assert rel_l2(Gg, Gref) <= 1e-4


def test_rr_tau_adj_replaces_tau0_in_adjoint_only():
    Gg, Gref, _, _, st = _window_gpu_vs_oracle(9, (300, 24, 1), 0.1, H.FP64, oobj.DISS, oadj.FTA,
                                               tau_adj=0.9)
    assert rel_l2(Gg, Gref) <= 1e-9


def test_rr_option_errors_and_checkpoint():
    P, d, R = _case(9, (200, 16, 1), 0.1)
    a = _solver(P, R, H.FP32)
    a.set_porosity(d)
    # the tangent-linear step is BGK only
    with pytest.raises(H.HlbmError) as e:
        H.hlbm_run_tangent(a.ctx, 3, np.zeros(P.dims[0] * P.dims[1]), H.OBJ_DISSIPATION)
    assert e.value.status == H.EINVAL
    # the collision cannot change on a live context
    opt = a.opt
    opt.collision = H.COLL_BGK
    with pytest.raises(H.HlbmError):
        H.hlbm_configure(a.ctx, P.tau0, P.Cs, opt)
    opt.collision = H.COLL_RR
    a.run_primal(101, 0)
    path = os.path.join(tempfile.mkdtemp(), "rr.bin")
    a.run_primal(60, 30)
    a.save(path)
    a.run_primal(50, 10)
    fa = a.field(H.FIELD_F)
    b = _solver(P, R, H.FP32)
    b.load(path)
    b.run_primal(50, 10)
    assert np.array_equal(b.field(H.FIELD_F), fa)
    # a BGK context refuses an RR checkpoint (different averages)
    c = Solver(P.q, P.dims, P.tau0, P.Cs, storage=H.FP32, u_in=P.u_in, regions=R)
    with pytest.raises(H.HlbmError):
        c.load(path)
    a.close()
    b.close()
    c.close()
