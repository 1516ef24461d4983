"""Pins of the oracle's recursive regularised collision (Sec. 2.2, Eq.
HRRLBM) and of its linearisation: Hermite moments of the third-order
equilibrium, the moments the collision relaxes, idempotence of the
regularisation, the tau = 1 and shear-wave special cases, complex-step
Jacobians against central differences, and the steady adjoint gradient
against central differences of J."""
import math

import numpy as np
import pytest

from oracle import adjoint as adj
from oracle import hlbm
from oracle import objectives as obj
from oracle.hlbm import Params
from oracle.lattice import CS2
from workloads import Regions, cylinder_porosity


def _state(P, seed, amp=0.02):
    rng = np.random.default_rng(seed)
    rho = 1.0 + 0.03 * rng.standard_normal(P.shape)
    u = 0.05 * rng.standard_normal((3,) + P.shape)
    if P.q == 9:
        u[2] = 0.0
    f = hlbm.equilibrium(rho, u, P)
    f = f * (1.0 + amp * rng.standard_normal(f.shape))
    d = rng.uniform(0.0, 1.0, P.shape)
    return f, d


def _small(q, Cs, tau0=0.62):
    dims = (8, 5, 4) if q == 19 else (9, 6, 1)
    return Params(q, dims, tau0=tau0, Cs=Cs, u_in=0.05, collision="rr")


@pytest.mark.parametrize("q", [9, 19])
def test_third_order_equilibrium_hermite_moments(q):
    P = _small(q, 0.0)
    rng = np.random.default_rng(1)
    rho = 1.0 + 0.05 * rng.standard_normal(P.shape)
    ut = 0.08 * rng.standard_normal((3,) + P.shape)
    if q == 9:
        ut[2] = 0.0
    feq = hlbm.equilibrium3(rho, ut, P)
    xi = P.xif
    assert np.abs(feq.sum(0) - rho).max() < 1e-15
    assert np.abs(np.einsum("ia,i...->a...", xi, feq) - rho * ut).max() < 1e-15
    # sum_i H2_i feq_i = rho u~ u~ (the third-order part adds nothing to second moments)
    a2 = np.einsum("iab,i...->ab...", P.H2, feq)
    assert np.abs(a2 - rho * np.einsum("a...,b...->ab...", ut, ut)).max() < 1e-15
    if q == 9:
        # D2Q9 represents H_xxy and H_xyy exactly: their projections are rho u~^3
        x, y = ut[0], ut[1]
        assert np.abs(np.einsum("i,i...->...", P.H3[:, 0, 0, 1], feq) - rho * x * x * y).max() < 1e-15
        assert np.abs(np.einsum("i,i...->...", P.H3[:, 0, 1, 1], feq) - rho * x * y * y).max() < 1e-15
        # and the third-order correction is w_i rho (9/2) (xi.u~) ((xi.u~)^2 - u~.u~)
        cu = np.einsum("ia,a...->i...", xi, ut)
        corr = P.w[:, None, None, None] * rho * 4.5 * cu * (cu * cu - (ut * ut).sum(0))
        assert np.abs(feq - hlbm.equilibrium(rho, ut, P) - corr).max() < 1e-16


@pytest.mark.parametrize("q,Cs", [(9, 0.0), (9, 0.2), (19, 0.1)])
def test_rr_collision_relaxes_the_bgk_moments(q, Cs):
    # mass kept; momentum rho u~ + (1 - omega) (j - rho u~); the stress relaxed
    # like BGK: sum xi xi f* = sum xi xi f^eq + (1 - omega) Pi_neq
    P = _small(q, Cs)
    f, d = _state(P, 3)
    fs, s = hlbm.collide(f, d, P)
    om = 1.0 / s["tau"]
    xi = P.xif
    assert np.abs(fs.sum(0) - f.sum(0)).max() < 1e-15
    j = np.einsum("ia,i...->a...", xi, f)
    rut = s["rho"] * s["ut"]
    assert np.abs(np.einsum("ia,i...->a...", xi, fs) - (rut + (1 - om) * (j - rut))).max() < 1e-15
    M2 = np.einsum("ia,ib,i...->ab...", xi, xi, fs)
    M2eq = np.einsum("ia,ib,i...->ab...", xi, xi, s["feq"])
    assert np.abs(M2 - (M2eq + (1 - om) * s["Pi"])).max() < 1e-15


@pytest.mark.parametrize("q", [9, 19])
def test_regularisation_is_idempotent(q):
    # a state already of the form f^eq(rho, u) + f^(1) relaxes to f^eq + (1 - 1/tau) f^(1)
    P = _small(q, 0.0, tau0=0.7)
    rng = np.random.default_rng(5)
    rho = 1.0 + 0.03 * rng.standard_normal(P.shape)
    u = 0.05 * rng.standard_normal((3,) + P.shape)
    if q == 9:
        u[2] = 0.0
    feq = hlbm.equilibrium3(rho, u, P)
    noise = 1e-3 * rng.standard_normal(feq.shape) * P.w[(slice(None),) + (None,) * 3]
    # remove mass and momentum from the non-equilibrium part
    noise -= P.w[:, None, None, None] * noise.sum(0)[None]
    mom = np.einsum("ia,i...->a...", P.xif, noise)
    noise -= P.w[:, None, None, None] * np.einsum("ia,a...->i...", P.xif, mom) / CS2
    assert np.abs(noise.sum(0)).max() < 1e-17
    assert np.abs(np.einsum("ia,i...->a...", P.xif, noise)).max() < 1e-17
    f1 = hlbm.regularised_noneq(noise, u, P)
    d = np.ones(P.shape)
    fs = hlbm.collide_rr(feq + f1, d, P, tau=np.full(P.shape, 0.7))
    assert np.abs(fs - (feq + (1 - 1 / 0.7) * f1)).max() < 1e-15


def test_third_order_noneq_coefficient_is_recursive_on_d2q9():
    P = _small(9, 0.0)
    rng = np.random.default_rng(8)
    fneq = 1e-3 * rng.standard_normal((9,) + P.shape)
    ut = 0.05 * rng.standard_normal((3,) + P.shape)
    ut[2] = 0.0
    f1 = hlbm.regularised_noneq(fneq, ut, P)
    a2 = np.einsum("iab,i...->ab...", P.H2, fneq)
    # a1^(3)_xxy = 2 u~_x a2_xy + u~_y a2_xx, a1^(3)_xyy = u~_x a2_yy + 2 u~_y a2_xy
    want_xxy = 2 * ut[0] * a2[0, 1] + ut[1] * a2[0, 0]
    want_xyy = ut[0] * a2[1, 1] + 2 * ut[1] * a2[0, 1]
    assert np.abs(np.einsum("i,i...->...", P.H3[:, 0, 0, 1], f1) - want_xxy).max() < 1e-17
    assert np.abs(np.einsum("i,i...->...", P.H3[:, 0, 1, 1], f1) - want_xyy).max() < 1e-17
    # orders 0-2 are the projections of f^neq
    assert np.abs(f1.sum(0) - fneq.sum(0)).max() < 1e-17
    assert np.abs(np.einsum("iab,i...->ab...", P.H2, f1) - a2).max() < 1e-17


@pytest.mark.parametrize("q", [9, 19])
def test_tau_one_gives_the_third_order_equilibrium(q):
    P = _small(q, 0.0, tau0=1.0)
    f, d = _state(P, 9)
    fs, s = hlbm.collide(f, d, P)
    assert np.abs(fs - hlbm.equilibrium3(s["rho"], s["ut"], P)).max() < 1e-16


def test_rr_shear_wave_recovers_viscosity():
    # the regularised collision keeps nu = c_s^2 (tau - 1/2) (Sec. 2.2)
    ny = 32
    P = Params(9, (200, ny, 1), tau0=0.8, u_in=0.0, collision="rr")
    k = 2 * math.pi / ny
    y = np.arange(ny)
    u = np.zeros((3,) + P.shape)
    A = 1e-3
    u[0] = A * np.sin(k * y)[None, :, None]
    f = hlbm.equilibrium(np.ones(P.shape), u, P)
    d = np.ones(P.shape)
    n = 60
    amps = []
    for t in range(n + 1):
        _, un = hlbm.moments(f, P)
        core = un[0][0, :, 80:120]
        amps.append(float((core * np.sin(k * y)[:, None]).sum() / (np.sin(k * y) ** 2).sum() / 40))
        f = hlbm.step(f, d, P)
    rate = -np.polyfit(np.arange(10, n + 1), np.log(amps[10:]), 1)[0]
    nu = CS2 * (P.tau0 - 0.5)
    assert abs(rate / (nu * k * k) - 1.0) < 5e-3


def _fd(fun, x, v, h):
    return (8 * (fun(x + h * v) - fun(x - h * v)) - (fun(x + 2 * h * v) - fun(x - 2 * h * v))) / (12 * h)


@pytest.mark.parametrize("q,Cs,mode", [(9, 0.0, adj.EXACT), (9, 0.3, adj.EXACT), (9, 0.3, adj.FTA),
                                       (19, 0.15, adj.EXACT)])
def test_rr_jacobians_vs_central_fd(q, Cs, mode):
    P = _small(q, Cs)
    f, d = _state(P, 21, amp=0.05)
    tt = np.random.default_rng(2).uniform(0.0, 0.05, P.shape) if mode == adj.FTA else None
    JC, Cd = adj.collision_jacobians(f, d, P, mode, None, tt)

    def C(ff, dd):
        if mode == adj.FTA:
            return hlbm.collide_rr(ff, dd, P, tau=P.tau0 + tt)
        return hlbm.collide(ff, dd, P)[0]

    rng = np.random.default_rng(4)
    v = rng.standard_normal(f.shape)
    fd = _fd(lambda x: C(x, d), f, v, 1e-5)
    an = np.einsum("ij...,j...->i...", JC, v)
    assert np.abs(fd - an).max() <= 1e-9 * max(1.0, np.abs(an).max())
    w = rng.standard_normal(d.shape)
    fdd = _fd(lambda x: C(f, x), d, w, 1e-5)
    assert np.abs(fdd - Cd * w).max() <= 1e-9 * max(1.0, np.abs(Cd).max())


def test_rr_with_bgk_jacobian_differs():
    # the two collisions have different Jacobians (guards against a dispatch
    # that silently falls back to BGK)
    P = _small(9, 0.0)
    f, d = _state(P, 2, amp=0.05)
    J_rr, _ = adj.collision_jacobians(f, d, P)
    Pb = Params(9, P.dims, tau0=P.tau0, Cs=0.0, u_in=P.u_in)
    J_bgk, _ = adj.collision_jacobians(f, d, Pb)
    assert np.abs(J_rr - J_bgk).max() > 1e-3


def _tiny(q, Cs):
    dims = (24, 12, 1) if q == 9 else (14, 8, 4)
    P = Params(q, dims, tau0=0.8, Cs=Cs, u_in=0.04, collision="rr")
    d = cylinder_porosity(dims, 7.0, dims[1] / 2.0, 2.0, 1.2, jitter=0.01, seed=3)
    nx, ny, nz = dims
    R = Regions(ffa_x=nx - 5, ffa_y=(0, ny), ffa_z=(0, nz),
                diss_box=(2, nx - 3, 0, ny, 0, nz), design_box=(0, nx, 0, ny, 0, nz))
    return P, d, R


@pytest.mark.parametrize("q,Cs", [(9, 0.0), (9, 0.2), (19, 0.0)])
@pytest.mark.parametrize("objective", [obj.FFA, obj.DISS])
def test_rr_steady_gradient_vs_central_fd(q, Cs, objective):
    P, d, R = _tiny(q, Cs)
    f = hlbm.initial_state(P)
    for _ in range(300):
        f = hlbm.step(f, d, P)
    f, res = adj.newton_steady(f, d, P)
    assert res < 1e-13
    g, gd = obj.partials(f, d, P, objective, R)
    lin = adj.Linearisation(f, d, P, adj.EXACT)
    G = adj.gradient(lin, adj.solve_adjoint_direct(lin, g), gd)

    def J_of(dd):
        ff, r = adj.newton_steady(f, dd, P, iters=10)
        assert r < 1e-13
        return obj.value(ff, dd, P, objective, R)

    rng = np.random.default_rng(17)
    h = 1e-5
    for _ in range(2):
        v = rng.standard_normal(d.shape)
        fd = (J_of(d + h * v) - J_of(d - h * v)) / (2 * h)
        an = float((G * v).sum())
        assert abs(fd - an) <= 2e-6 * max(abs(an), 1e-3 * np.abs(G).sum())
