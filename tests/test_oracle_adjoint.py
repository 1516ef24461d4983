"""Pins of the oracle's derivatives, adjoint and gradient against central
finite differences of the primal, sparse direct solves, the duality
identity and the special cases the paper's method reduces to."""
import numpy as np
import pytest

from oracle import adjoint as adj
from oracle import hlbm
from oracle import meanflow
from oracle import objectives as obj
from oracle.hlbm import Params
from workloads import Regions, cylinder_porosity


def _state(P, seed, amp=0.02):
    rng = np.random.default_rng(seed)
    rho = 1.0 + 0.03 * rng.standard_normal(P.shape)
    u = 0.04 * rng.standard_normal((3,) + P.shape)
    if P.q == 9:
        u[2] = 0.0
    f = hlbm.equilibrium(rho, u, P)
    f = f * (1.0 + amp * rng.standard_normal(f.shape))
    d = rng.uniform(0.0, 1.0, P.shape)
    return f, d


def _small(q, Cs):
    dims = (8, 5, 4) if q == 19 else (9, 6, 1)
    return Params(q, dims, tau0=0.62, Cs=Cs, u_in=0.05)


def _regions(P):
    nx, ny, nz = P.dims
    return Regions(ffa_x=nx - 3, ffa_y=(0, ny), ffa_z=(0, nz),
                   diss_box=(1, nx - 1, 0, ny, 0, nz), design_box=(0, nx, 0, ny, 0, nz))


def _fd(fun, x, v, h):
    """Fourth-order central difference of fun along v."""
    return (8 * (fun(x + h * v) - fun(x - h * v)) - (fun(x + 2 * h * v) - fun(x - 2 * h * v))) / (12 * h)


@pytest.mark.parametrize("q,Cs", [(9, 0.0), (9, 0.2), (19, 0.1)])
@pytest.mark.parametrize("objective", [obj.FFA, obj.DISS])
def test_objective_partials_vs_central_fd(q, Cs, objective):
    P = _small(q, Cs)
    R = _regions(P)
    f, d = _state(P, 11)
    g, gd = obj.partials(f, d, P, objective, R)
    rng = np.random.default_rng(2)
    for _ in range(3):
        v = rng.standard_normal(f.shape)
        fd = _fd(lambda x: obj.value(x, d, P, objective, R), f, v, 1e-6)
        an = float((g * v).sum())
        assert abs(fd - an) <= 1e-7 * max(1.0, abs(an))
        w = rng.standard_normal(d.shape)
        fdd = _fd(lambda x: obj.value(f, x, P, objective, R), d, w, 1e-6)
        assert abs(fdd - float((gd * w).sum())) <= 1e-7 * max(1.0, abs(fdd))


@pytest.mark.parametrize("q,Cs", [(9, 0.0), (9, 0.3), (19, 0.15)])
def test_collision_jacobians_vs_central_fd(q, Cs):
    P = _small(q, Cs)
    f, d = _state(P, 4, amp=0.05)
    JC, Cd = adj.collision_jacobians(f, d, P, adj.EXACT)
    rng = np.random.default_rng(9)
    for _ in range(3):
        v = rng.standard_normal(f.shape)
        fd = _fd(lambda x: hlbm.collide(x, d, P)[0], f, v, 1e-5)
        an = np.einsum("ij...,j...->i...", JC, v)
        assert np.abs(fd - an).max() < 1e-7 * np.abs(an).max()
        w = rng.standard_normal(d.shape)
        fdd = _fd(lambda x: hlbm.collide(f, x, P)[0], d, w, 1e-5)
        assert np.abs(fdd - Cd * w).max() < 1e-7 * np.abs(Cd * w).max()


def test_fta_is_bgk_jacobian_with_frozen_tau():
    # Sec. 5.4: FTA drops d tau_turb/df and uses the averaged tau_turb
    P = _small(9, 0.25)
    f, d = _state(P, 6)
    tt = 0.037
    JF, CdF = adj.collision_jacobians(f, d, P, adj.FTA, tau_t_bar=np.full(P.shape, tt))
    Pb = Params(9, P.dims, tau0=P.tau0 + tt, Cs=0.0, u_in=P.u_in)
    JB, CdB = adj.collision_jacobians(f, d, Pb, adj.EXACT)
    assert np.abs(JF - JB).max() < 1e-15 and np.abs(CdF - CdB).max() < 1e-15


def test_cs_zero_exact_equals_fta():
    P = _small(19, 0.0)
    f, d = _state(P, 8)
    JE, CdE = adj.collision_jacobians(f, d, P, adj.EXACT)
    JF, CdF = adj.collision_jacobians(f, d, P, adj.FTA, tau_t_bar=np.zeros(P.shape))
    assert np.abs(JE - JF).max() == 0 and np.abs(CdE - CdF).max() == 0


@pytest.mark.parametrize("q,Cs", [(9, 0.0), (9, 0.2), (19, 0.1)])
def test_step_jacobian_vs_central_fd(q, Cs):
    # A = dPhi/df and dPhi/dd of one whole step (collision, streaming and the
    # inflow/outflow nodes) against central differences of hlbm.step
    P = _small(q, Cs)
    f, d = _state(P, 21, amp=0.06)   # keeps ||Pi|| away from its kink at 0
    f = hlbm.apply_boundary(f, P)
    lin = adj.Linearisation(f, d, P, adj.EXACT, outlet="streamed")
    rng = np.random.default_rng(5)
    for _ in range(3):
        v = rng.standard_normal(f.shape)
        fd = _fd(lambda x: hlbm.step(x, d, P), f, v, 1e-6)
        an = lin.jvp(v)
        assert np.abs(fd - an).max() < 1e-7 * np.abs(an).max()
        w = rng.standard_normal(d.shape)
        fdd = _fd(lambda x: hlbm.step(f, x, P), d, w, 1e-6)
        an = (lin.D @ w.ravel()).reshape(f.shape)
        assert np.abs(fdd - an).max() < 1e-7 * np.abs(an).max()
    # transposition: <w, A v> = <A^T w, v>
    v = rng.standard_normal(f.shape)
    w = rng.standard_normal(f.shape)
    lhs = float((w * lin.jvp(v)).sum())
    rhs = float((lin.vjp(w) * v).sum())
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


def test_streaming_matrix_matches_stream():
    for q, dims in ((9, (7, 5, 1)), (19, (6, 4, 3))):
        P = Params(q, dims, tau0=0.6)
        v = np.random.default_rng(0).standard_normal((q,) + P.shape)
        S = adj.streaming_matrix(P)
        assert np.abs((S @ v.ravel()).reshape(v.shape) - hlbm.stream(v, P)).max() == 0


def _tiny_case(q=9, Cs=0.0, tau0=0.8, sym=False):
    if q == 9:
        dims = (24, 12, 1)
    else:
        dims = (14, 8, 4)
    P = Params(q, dims, tau0=tau0, Cs=Cs, u_in=0.04)
    d = cylinder_porosity(dims, 7.0, dims[1] / 2.0, 2.0, 1.2, jitter=0.0 if sym else 0.01, seed=3)
    nx, ny, nz = dims
    R = Regions(ffa_x=nx - 5, ffa_y=(0, ny), ffa_z=(0, nz),
                diss_box=(2, nx - 3, 0, ny, 0, nz), design_box=(0, nx, 0, ny, 0, nz))
    return P, d, R


def _steady(P, d, steps=300):
    f = hlbm.initial_state(P)
    for _ in range(steps):
        f = hlbm.step(f, d, P)
    f, res = adj.newton_steady(f, d, P)
    assert res < 1e-13
    return f


@pytest.mark.parametrize("q,Cs", [(9, 0.0), (9, 0.2), (19, 0.0)])
@pytest.mark.parametrize("objective", [obj.FFA, obj.DISS])
def test_steady_gradient_vs_central_fd(q, Cs, objective):
    # Eq. gradients_steady: dJ/dd from the steady adjoint matches central
    # differences of J at the perturbed steady states (directional and per cell)
    P, d, R = _tiny_case(q, Cs)
    f = _steady(P, d)
    g, gd = obj.partials(f, d, P, objective, R)
    lin = adj.Linearisation(f, d, P, adj.EXACT)
    lam, it, r = adj.solve_adjoint(lin, g, tol=1e-13, max_iter=200000)
    assert r <= 1e-13
    G = adj.gradient(lin, lam, gd)

    def J_of(dd):
        return obj.value(_steady_from(f, dd, P), dd, P, objective, R)

    rng = np.random.default_rng(17)
    h = 1e-5
    for _ in range(2):
        v = rng.standard_normal(d.shape)
        fd = (J_of(d + h * v) - J_of(d - h * v)) / (2 * h)
        an = float((G * v).sum())
        assert abs(fd - an) <= 2e-6 * max(abs(an), 1e-3 * np.abs(G).sum())


def _steady_from(f, d, P):
    f, res = adj.newton_steady(f, d, P, iters=10)
    assert res < 1e-13
    return f


def test_adjoint_iteration_matches_direct_solve_and_duality():
    # fixed point of lambda <- A^T lambda + g solves (I - A^T) lambda = g;
    # duality <lambda, (I - A) v> = <g, v>
    P, d, R = _tiny_case(9, 0.0)
    f = _steady(P, d)
    g, _ = obj.partials(f, d, P, obj.DISS, R)
    lin = adj.Linearisation(f, d, P, adj.EXACT)
    lam_it, it, r = adj.solve_adjoint(lin, g, tol=1e-13, max_iter=200000)
    lam_dir = adj.solve_adjoint_direct(lin, g)
    assert np.abs(lam_it - lam_dir).max() <= 1e-10 * np.abs(lam_dir).max()
    v = np.random.default_rng(1).standard_normal(f.shape)
    lhs = float((lam_dir * (v - lin.jvp(v))).sum())
    rhs = float((g * v).sum())
    assert abs(lhs - rhs) <= 1e-10 * abs(rhs)


def test_window_one_is_steady_state_sample():
    # avg_window = 1: f_bar is the last canonical state sampled
    P, d, R = _tiny_case(9, 0.0)
    f0 = hlbm.initial_state(P)
    out = meanflow.run_primal(f0, d, P, 20, 1, R)
    f = f0
    for _ in range(19):
        f = hlbm.step(f, d, P)
    assert np.abs(out["fbar"] - f).max() == 0
    assert np.abs(out["f"] - hlbm.step(f, d, P)).max() == 0
    assert out[("Jbar", obj.FFA)] == obj.value(f, d, P, obj.FFA, R)


def test_mean_of_window_matches_stored_history():
    # tracking average (Eq. averageObjective) against an explicit history
    P, d, R = _tiny_case(9, 0.1)
    f = hlbm.initial_state(P)
    hist, Js, gs = [], [], []
    for n in range(12):
        if n >= 7 and (n - 7) % 2 == 0:
            hist.append(f)
            Js.append(obj.value(f, d, P, obj.DISS, R))
            gs.append(obj.partials(f, d, P, obj.DISS, R)[0])
        f = hlbm.step(f, d, P)
    out = meanflow.run_primal(hlbm.initial_state(P), d, P, 12, 5, R, obj.DISS, stride=2)
    assert out["nsamples"] == 3
    assert np.abs(out["fbar"] - np.mean(hist, axis=0)).max() < 1e-16
    assert abs(out[("Jbar", obj.DISS)] - np.mean(Js)) < 1e-15
    assert np.abs(out[("gbar", obj.DISS)] - np.mean(gs, axis=0)).max() < 1e-16


def test_symmetric_geometry_gives_symmetric_gradient():
    # a porosity field symmetric about y = ny/2 gives G(x, y) = G(x, ny - y)
    P, d, R = _tiny_case(9, 0.0, sym=True)
    f = _steady(P, d)
    g, gd = obj.partials(f, d, P, obj.DISS, R)
    lin = adj.Linearisation(f, d, P, adj.EXACT)
    G = adj.gradient(lin, adj.solve_adjoint_direct(lin, g), gd)
    ny = P.dims[1]
    refl = G[:, (-np.arange(ny)) % ny, :]
    assert np.abs(G - refl).max() <= 1e-10 * np.abs(G).max()


def test_mea_surface_nodes_and_linearity():
    # Sec. 4.1: J_MEA is linear in f, so its derivative is exact under any
    # finite difference; surface nodes are fluid cells next to solid ones
    P, d, R = _tiny_case(9, 0.0, sym=True)
    surf = obj.surface_nodes(d, P)
    assert surf.sum() > 0 and not (surf & (d < 0.5)).any()
    f, _ = _state(P, 31)
    g, gd = obj.partials(f, d, P, obj.MEA, R)
    assert np.abs(gd).max() == 0
    rng = np.random.default_rng(3)
    v = rng.standard_normal(f.shape)
    lhs = obj.value(f + 0.37 * v, d, P, obj.MEA, R) - obj.value(f, d, P, obj.MEA, R)
    assert abs(lhs - 0.37 * float((g * v).sum())) <= 1e-12 * max(1.0, abs(lhs))
    # a uniform flow past no body exerts no force
    Pe = Params(9, P.dims, tau0=0.8, u_in=0.04)
    assert obj.mea_value(hlbm.initial_state(Pe), np.ones(P.shape), Pe) == 0.0


def test_mea_steady_gradient_vs_central_fd():
    P, d, R = _tiny_case(9, 0.0)
    f = _steady(P, d)
    g, gd = obj.partials(f, d, P, obj.MEA, R)
    lin = adj.Linearisation(f, d, P, adj.EXACT)
    G = adj.gradient(lin, adj.solve_adjoint_direct(lin, g), gd)
    rng = np.random.default_rng(23)
    v = rng.standard_normal(d.shape) * (np.abs(d - 0.5) > 0.1)   # keep the surface set fixed
    h = 1e-6
    Jp = obj.value(_steady_from(f, d + h * v, P), d + h * v, P, obj.MEA, R)
    Jm = obj.value(_steady_from(f, d - h * v, P), d - h * v, P, obj.MEA, R)
    fd = (Jp - Jm) / (2 * h)
    an = float((G * v).sum())
    assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-6)


@pytest.mark.parametrize("q,Cs,mode,collision", [(9, 0.0, adj.EXACT, "bgk"), (9, 0.2, adj.EXACT, "bgk"),
                                                 (19, 0.15, adj.EXACT, "bgk"), (19, 0.15, adj.FTA, "bgk"),
                                                 (19, 0.1, adj.EXACT, "rr")])
def test_matrix_free_linearisation_is_the_assembled_one(q, Cs, mode, collision):
    # the factor-by-factor form (per-cell blocks, B S sparse) applies the same
    # maps as the assembled matrices that the central-difference pins check
    P = Params(q, (10, 6, 4) if q == 19 else (12, 7, 1), tau0=0.58, Cs=Cs, u_in=0.05,
               collision=collision)
    f, d = _state(P, 31, amp=0.05)
    f = hlbm.apply_boundary(f, P)
    tt = np.full(P.shape, 0.021)
    A = adj.Linearisation(f, d, P, mode, tau_adj=0.63, tau_t_bar=tt)
    M = adj.Linearisation(f, d, P, mode, tau_adj=0.63, tau_t_bar=tt, assemble=False)
    rng = np.random.default_rng(2)
    v = rng.standard_normal(f.shape)
    w = rng.standard_normal(f.shape)
    for a, b in ((A.jvp(v), M.jvp(v)), (A.vjp(w), M.vjp(w)), (A.dd_vjp(w), M.dd_vjp(w))):
        assert np.abs(a - b).max() <= 1e-13 * np.abs(a).max()
    g = rng.standard_normal(f.shape)
    la, ka, ra = adj.solve_adjoint(A, g, tol=0.0, max_iter=7)
    lm, km, rm = adj.solve_adjoint(M, g, tol=0.0, max_iter=7)
    assert ka == km == 7 and abs(ra - rm) <= 1e-12 * ra
    assert np.abs(la - lm).max() <= 1e-12 * np.abs(la).max()
    gd = rng.standard_normal(d.shape)
    Ga, Gm = adj.gradient(A, la, gd), adj.gradient(M, lm, gd)
    assert np.abs(Ga - Gm).max() <= 1e-12 * np.abs(Ga).max()
