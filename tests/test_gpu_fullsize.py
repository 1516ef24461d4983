"""Parity at the benchmark workloads' full sizes, in the launch configuration
the benchmark uses, on outputs the oracle can compute directly.

* Kármán case (D2Q9 1100x410, FP32): primal steps, an averaging step, and
  adjoint iterations from the same state, compared element by element over
  the whole grid (the oracle does one step of this grid in well under a
  second).
* Steady Re-20 case (D2Q9 200x80, FP64): the whole of Algorithm 1 at its full
  size, gradient compared with the oracle's direct adjoint solve.
* LES case (D3Q19 640x320x100, FP32 and FP16 deviations): one primal step
  checked on sampled sub-boxes, which the oracle recomputes from the same
  state with a one-cell halo.
"""
import numpy as np
import pytest

from oracle import adjoint as oadj
from oracle import hlbm as ohlbm
from oracle import meanflow as omf
from oracle import objectives as oobj
from tests.hlbm_cases import direction_perm, params_of, rel_l2, to_lib
from workloads import make_workload

pytestmark = pytest.mark.gpu

H = pytest.importorskip("paper_2606_31707_b300.hlbm")
from paper_2606_31707_b300 import Solver  # noqa: E402


def _state_near(P, wl, seed=5, amp=0.002):
    rng = np.random.default_rng(seed)
    u = np.zeros((3,) + P.shape)
    u[0] = wl.u0 * (1 + 0.1 * rng.standard_normal(P.shape))
    u[1] = 0.1 * wl.u0 * rng.standard_normal(P.shape)
    if P.q == 19:
        u[2] = 0.1 * wl.u0 * rng.standard_normal(P.shape)
    f = ohlbm.equilibrium(np.ones(P.shape), u, P) * (1 + amp * rng.standard_normal((P.q,) + P.shape))
    return ohlbm.apply_boundary(f, P)


def test_karman_fullsize_primal_average_and_adjoint_iterations():
    wl = make_workload("karman2d_re100")
    P = params_of(wl)
    f0 = _state_near(P, wl)
    s = Solver(9, wl.dims, P.tau0, 0.0, storage=H.FP32, u_in=wl.u0, regions=wl.regions)
    perm = direction_perm(s.xi, P)
    s.set_porosity(wl.porosity)
    s.set_field(H.FIELD_F, to_lib(f0, perm))
    s.run_primal(3, 0)
    f = f0
    for _ in range(3):
        f = ohlbm.step(f, wl.porosity, P)
    assert rel_l2(s.field(H.FIELD_F), to_lib(f, perm)) <= 1e-6
    # one averaging step from the state reached
    s.set_field(H.FIELD_F, to_lib(f, perm))
    s.run_primal(1, 1)
    out = omf.run_primal(f, wl.porosity, P, 1, 1, wl.regions, 3)
    for o, gf in ((oobj.FFA, H.FIELD_GBAR_FFA), (oobj.DISS, H.FIELD_GBAR_DISS)):
        assert rel_l2(s.field(gf), to_lib(out[("gbar", o)], perm)) <= 1e-5
        assert abs(s.objective(o) - out[("Jbar", o)]) <= 1e-5 * abs(out[("Jbar", o)])
    # 20 adjoint iterations from zero on both sides, same averaged state
    lin = oadj.Linearisation(out["fbar"], wl.porosity, P, oadj.EXACT)
    for o in (oobj.FFA, oobj.DISS):
        st, it, res = s.solve_adjoint(o, H.ADJ_EXACT, 0.0, 20)
        assert it == 20
        lam, _, _ = oadj.solve_adjoint(lin, out[("gbar", o)], tol=0.0, max_iter=20)
        mu_ref = to_lib(lin.mu(lam), perm)
        assert rel_l2(s.field(H.FIELD_LAMBDA), mu_ref) <= 1e-5
        G = oadj.gradient(lin, lam, out[("dJdd_bar", o)])
        assert rel_l2(s.gradient(), G) <= 1e-5
    s.close()


def test_cylinder_re20_fullsize_fp64_algorithm1():
    # the whole of Algorithm 1 on each side from the same initial state: 6000
    # primal steps (window 1: f_bar is the state the last step starts from),
    # the steady adjoint and the gradient
    wl = make_workload("cyl2d_re20")
    P = params_of(wl)
    s = Solver(9, wl.dims, P.tau0, 0.0, storage=H.FP64, u_in=wl.u0, regions=wl.regions)
    s.set_porosity(wl.porosity)
    s.run_primal(wl.steps, 1)
    perm = direction_perm(s.xi, P)
    fbar = ohlbm.initial_state(P)
    for _ in range(wl.steps - 1):
        fbar = ohlbm.step(fbar, wl.porosity, P)
    out = omf.run_primal(fbar, wl.porosity, P, 1, 1, wl.regions, 3)
    # the GPU's primal agrees with the oracle's over the 6000 steps
    assert rel_l2(s.field(H.FIELD_F), to_lib(out["f"], perm)) <= 1e-12
    lin = oadj.Linearisation(fbar, wl.porosity, P, oadj.EXACT)
    for o in (oobj.FFA, oobj.DISS):
        st, it, res = s.solve_adjoint(o, H.ADJ_EXACT, 1e-10, 2_000_000)
        assert st == H.OK
        lam = oadj.solve_adjoint_direct(lin, out[("gbar", o)])
        G = oadj.gradient(lin, lam, out[("dJdd_bar", o)])
        assert rel_l2(s.gradient(), G) <= 1e-8
    s.close()


def _subbox_step(f, d, P, box):
    """One oracle step on the sub-box (x0, x1, y0, y1, z0, z1) of an interior
    region, computed from a one-cell halo of the given state."""
    x0, x1, y0, y1, z0, z1 = box
    sub = f[:, z0 - 1:z1 + 1, y0 - 1:y1 + 1, x0 - 1:x1 + 1]
    dsub = d[z0 - 1:z1 + 1, y0 - 1:y1 + 1, x0 - 1:x1 + 1]
    Ps = ohlbm.Params(P.q, (x1 - x0 + 2, y1 - y0 + 2, z1 - z0 + 2), tau0=P.tau0, Cs=P.Cs, u_in=P.u_in)
    fs, _ = ohlbm.collide(sub, dsub, Ps)
    st = ohlbm.stream(fs, Ps)
    return st[:, 1:-1, 1:-1, 1:-1]


@pytest.mark.parametrize("storage,tol", [(H.FP32, 1e-6), (H.FP16DEV, 2e-3)])
def test_les_fullsize_primal_step_on_sampled_boxes(storage, tol):
    wl = make_workload("les3d_re3900")
    P = params_of(wl)
    nx, ny, nz = wl.dims
    rng = np.random.default_rng(9)
    s = Solver(19, wl.dims, P.tau0, wl.Cs, storage=storage, u_in=wl.u0, regions=wl.regions)
    perm = direction_perm(s.xi, P)
    s.set_porosity(wl.porosity)
    # a non-equilibrium state built by the oracle's equilibrium: a seeded smooth
    # velocity field with 0.5 % population noise, written through the ABI
    u = np.zeros((3,) + P.shape)
    u[0] = wl.u0
    u[1] = 0.2 * wl.u0 * np.sin(2 * np.pi * np.arange(ny) / ny)[None, :, None]
    u[2] = 0.1 * wl.u0 * rng.standard_normal(P.shape)
    f = ohlbm.equilibrium(np.ones(P.shape), u, P)
    del u
    f *= 1.0 + 0.005 * rng.standard_normal(f.shape)
    f = ohlbm.apply_boundary(f, P)
    s.set_field(H.FIELD_F, to_lib(f, perm))
    s.run_primal(1, 0)
    g = s.field(H.FIELD_F)[np.argsort(perm)]
    boxes = [(150, 166, 150, 170, 40, 48), (300, 316, 10, 26, 3, 9), (600, 620, 290, 310, 90, 98)]
    for box in boxes:
        ref = _subbox_step(f, wl.porosity, P, box)
        x0, x1, y0, y1, z0, z1 = box
        assert rel_l2(g[:, z0:z1, y0:y1, x0:x1] - P.w[:, None, None, None],
                      ref - P.w[:, None, None, None]) <= tol
    s.close()


@pytest.mark.parametrize("mode", [oadj.EXACT, oadj.FTA])
def test_les_config_adjoint_iterations_kernel_level(mode):
    # the LES configuration (D3Q19, C_S = 0.1, tau0 from Re 3900, FP32) on a
    # reduced grid: 30 adjoint iterations and the gradient from the same
    # averaged state on both sides (exact LES and frozen turbulence, tau_adj 0.6)
    wl = make_workload("les3d_re3900_quarter")
    dims = (64, 24, 12)
    P = ohlbm.Params(19, dims, tau0=ohlbm.tau_from_reynolds(wl.u0, wl.L, wl.Re), Cs=wl.Cs, u_in=wl.u0)
    from workloads import Regions, cylinder_porosity
    d = cylinder_porosity(dims, 16.0, 12.0, 4.0, 2.0, jitter=0.01, seed=4)
    R = Regions(ffa_x=40, ffa_y=(0, 24), ffa_z=(0, 12), diss_box=(2, 60, 0, 24, 0, 12),
                design_box=(0, 64, 0, 24, 0, 12))
    f = _state_near(P, wl, seed=8, amp=0.01)
    s = Solver(19, dims, P.tau0, P.Cs, storage=H.FP32, u_in=wl.u0, regions=R, tau_adj=0.6)
    perm = direction_perm(s.xi, P)
    s.set_porosity(d)
    s.set_field(H.FIELD_F, to_lib(f, perm))
    s.run_primal(4, 3)
    out = omf.run_primal(f, d, P, 4, 3, R, 3)
    lin = oadj.Linearisation(out["fbar"], d, P, mode, 0.6, out["tau_t_bar"])
    for o in (oobj.FFA, oobj.DISS):
        st, it, res = s.solve_adjoint(o, mode, 0.0, 30)
        lam, _, _ = oadj.solve_adjoint(lin, out[("gbar", o)], tol=0.0, max_iter=30)
        assert rel_l2(s.field(H.FIELD_LAMBDA), to_lib(lin.mu(lam), perm)) <= 1e-4
        G = oadj.gradient(lin, lam, out[("dJdd_bar", o)])
        assert rel_l2(s.gradient(), G) <= 1e-4
    s.close()
