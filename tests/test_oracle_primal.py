"""Pins of the FP64 oracle's primal against what the paper and the
mathematics fix: lattice isotropy, equilibrium moments, collision
invariants, the Smagorinsky tau_eff definition, exact discrete Darcy decay,
the viscosity-relaxation relation (shear-wave decay), the plane-Poiseuille and
Brinkman porous-channel closed forms, and fixed points."""
import math

import numpy as np
import pytest

from oracle import hlbm
from oracle.hlbm import Params
from oracle.lattice import CS2, velocity_set


@pytest.mark.parametrize("q", [9, 19])
def test_lattice_moments_and_isotropy(q):
    # Sec. 2.1: DdQq velocity sets; weights give the Maxwellian moments
    xi, w, opp = velocity_set(q)
    xf = xi.astype(float)
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.abs(w @ xf).max() < 1e-15
    M2 = np.einsum("i,ia,ib->ab", w, xf, xf)
    dim = 2 if q == 9 else 3
    expect = np.zeros((3, 3))
    expect[:dim, :dim] = CS2 * np.eye(dim)
    assert np.abs(M2 - expect).max() < 1e-15
    M4 = np.einsum("i,ia,ib,ic,id->abcd", w, xf, xf, xf, xf)
    d = np.zeros((3, 3))
    d[:dim, :dim] = np.eye(dim)
    iso = CS2 ** 2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
                      + np.einsum("ad,bc->abcd", d, d))
    assert np.abs(M4 - iso).max() < 1e-15
    assert (xi[opp] == -xi).all()
    assert len({tuple(v) for v in xi}) == q


def _random_state(P, seed, amp=0.02):
    rng = np.random.default_rng(seed)
    shape = P.shape
    rho = 1.0 + 0.05 * rng.standard_normal(shape)
    u = 0.05 * rng.standard_normal((3,) + shape)
    if P.q == 9:
        u[2] = 0.0
    f = hlbm.equilibrium(rho, u, P)
    f = f * (1.0 + amp * rng.standard_normal(f.shape))
    d = rng.uniform(0.0, 1.0, shape)
    return f, d


@pytest.mark.parametrize("q", [9, 19])
def test_equilibrium_moments(q):
    # Eq. 3: the second-order equilibrium carries rho, rho u~ and
    # rho c_s^2 delta + rho u~ u~ exactly on these lattices
    P = Params(q, (5, 4, 3 if q == 19 else 1), tau0=0.6)
    rng = np.random.default_rng(1)
    rho = 1 + 0.1 * rng.standard_normal(P.shape)
    ut = 0.1 * rng.standard_normal((3,) + P.shape)
    if q == 9:
        ut[2] = 0
    feq = hlbm.equilibrium(rho, ut, P)
    assert np.abs(feq.sum(0) - rho).max() < 1e-14
    m = np.tensordot(P.xif.T, feq, axes=(1, 0))
    assert np.abs(m - rho * ut).max() < 1e-14
    M2 = np.einsum("ia,ib,i...->ab...", P.xif, P.xif, feq)
    dim = 2 if q == 9 else 3
    for a in range(dim):
        for b in range(dim):
            ref = rho * ut[a] * ut[b] + (CS2 * rho if a == b else 0.0)
            assert np.abs(M2[a, b] - ref).max() < 1e-14


@pytest.mark.parametrize("q,Cs", [(9, 0.0), (9, 0.3), (19, 0.1)])
def test_collision_invariants(q, Cs):
    # Eq. 2 with Eq. 3: mass is conserved; momentum changes by the Brinkman
    # term -rho (u - u~)/tau_eff = -rho (1-d)(u - u_s)/tau_eff
    P = Params(q, (6, 5, 4 if q == 19 else 1), tau0=0.7, Cs=Cs, u_s=(0.01, -0.02, 0.0))
    f, d = _random_state(P, 3)
    fs, s = hlbm.collide(f, d, P)
    assert np.abs((fs - f).sum(0)).max() < 1e-15
    dm = np.tensordot(P.xif.T, fs - f, axes=(1, 0))
    us = np.array(P.u_s).reshape(3, 1, 1, 1)
    expect = -s["rho"] * (1 - d) * (s["u"] - us) / s["tau"]
    if q == 9:
        expect[2] = 0
    assert np.abs(dm - expect).max() < 1e-15
    # at d = 1 momentum is conserved exactly
    fs1, _ = hlbm.collide(f, np.ones_like(d), P)
    assert np.abs(np.tensordot(P.xif.T, fs1 - f, axes=(1, 0))).max() < 1e-15


@pytest.mark.parametrize("Cs", [0.1, 0.17, 0.5])
def test_tau_eff_solves_smagorinsky_definition(Cs):
    # Sec. 2.2: tau_eff = (nu_mo + nu_turb)/c_s^2 + 1/2, nu_turb = (C_S dx)^2 |S|,
    # with S from the non-equilibrium stress at tau_eff (Sec. 4.3); |S| = sqrt(2 S:S)
    P = Params(19, (4, 4, 4), tau0=0.5012, Cs=Cs)
    f, d = _random_state(P, 5, amp=0.05)
    s = hlbm.local_state(f, d, P)
    tau = s["tau"]
    S = -s["Pi"] / (2 * tau * CS2)
    absS = np.sqrt(2 * np.einsum("ab...,ab...->...", S, S))
    nu_t = Cs ** 2 * absS
    nu_mo = CS2 * (P.tau0 - 0.5)
    assert np.abs(tau - ((nu_mo + nu_t) / CS2 + 0.5)).max() < 1e-14
    assert (tau >= P.tau0).all()


@pytest.mark.parametrize("dval", [0.0, 0.3, 0.9, 1.0])
def test_uniform_darcy_decay_closed_form(dval):
    # Brinkman term (Eq. 1, -nu/K u with nu/K = (1-d)/tau): a uniform state
    # with uniform d decays per step exactly by (1 - (1-d)/tau0); columns
    # that the inflow/outflow nodes have not reached yet stay uniform.
    P = Params(9, (40, 6, 1), tau0=0.8, u_in=0.05)
    u = np.zeros((3,) + P.shape)
    u[0], u[1] = 0.04, -0.01
    f = hlbm.equilibrium(np.ones(P.shape), u, P)
    d = np.full(P.shape, dval)
    n = 6
    for _ in range(n):
        f = hlbm.step(f, d, P)
    rho, un = hlbm.moments(f, P)
    core = slice(n + 1, P.dims[0] - n - 2)
    fac = (1 - (1 - dval) / P.tau0) ** n
    assert np.abs(un[0][..., core] - 0.04 * fac).max() < 1e-15
    assert np.abs(un[1][..., core] + 0.01 * fac).max() < 1e-15
    assert np.abs(rho[..., core] - 1.0).max() < 1e-14


def test_shear_wave_recovers_viscosity():
    # Sec. 2.1: nu = c_s^2 (tau - 1/2).  A transverse shear wave
    # u_x = A sin(k y) decays like exp(-nu k^2 t) (Navier-Stokes limit of
    # Eq. 2, up to O(k^2) lattice error).  Checked far from the inflow and
    # outflow columns over fewer steps than they need to reach the core.
    ny = 32
    P = Params(9, (200, ny, 1), tau0=0.8, u_in=0.0)
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


@pytest.mark.parametrize("q", [9, 19])
def test_uniform_flow_is_fixed_point_without_body(q):
    # d = 1 everywhere: the inflow equilibrium is a fixed point of the step
    P = Params(q, (12, 6, 4 if q == 19 else 1), tau0=0.6, Cs=0.1 if q == 19 else 0.0, u_in=0.05)
    f0 = hlbm.initial_state(P)
    f1 = hlbm.step(f0, np.ones(P.shape), P)
    assert np.abs(f1 - f0).max() < 1e-15


def test_tau_from_reynolds_matches_configs():
    # Re = u D / nu (Sec. 5) with nu = c_s^2 (tau - 1/2) (Sec. 2.1)
    assert abs(hlbm.tau_from_reynolds(0.05, 20, 20) - 0.65) < 1e-15
    assert abs(hlbm.tau_from_reynolds(0.04, 50, 100) - 0.56) < 1e-15
    assert abs(hlbm.tau_from_reynolds(0.05, 60, 40) - 0.725) < 1e-15


def _channel_steady(dp, tau=1.0, ny=9, nx=64, u_in=0.02):
    """Steady flow through a y-periodic channel whose row y = 0 is solid
    (d = 0, so the walls sit at y = 0 and y = ny) filled with porosity dp,
    driven by the uniform inflow; returns the profile u_x(y) and the
    pressure gradient (1/rho) dp/dx in the middle of the channel."""
    from oracle import adjoint as adj
    P = Params(9, (nx, ny, 1), tau0=tau, u_in=u_in)
    d = np.full(P.shape, dp)
    d[0, 0, :] = 0.0
    f = hlbm.initial_state(P)
    for _ in range(200):
        f = hlbm.step(f, d, P)
    f, res = adj.newton_steady(f, d, P, iters=12)
    assert res < 1e-13
    rho, u = hlbm.moments(f, P)
    x0 = nx // 2
    prof = u[0, 0, :, x0].copy()
    prof[0] = 0.0  # the solid row is the wall node, not channel flow
    G = CS2 * (rho[0, 1:, x0 + 5] - rho[0, 1:, x0 - 5]).mean() / 10 / rho[0, 1:, x0].mean()
    return prof, G, P


def test_plane_poiseuille_closed_form():
    # Sec. 2.1 in a channel: with tau = 1 a solid (d = 0) row relaxes to rest
    # each step, a no-slip node.  Fully developed, nu u'' = (1/rho) dp/dx, so
    # u = A y (H - y) with -2 nu A = (1/rho) dp/dx.
    prof, G, P = _channel_steady(1.0)
    H = P.dims[1]
    y = np.arange(H)
    para = y * (H - y)
    A = (prof * para).sum() / (para ** 2).sum()
    assert np.abs(prof - A * para).max() <= 1e-4 * np.abs(A * para).max()
    assert abs(-2 * P.nu0 * A / G - 1.0) <= 1e-3


@pytest.mark.parametrize("dp", [0.97, 0.9, 0.7])
def test_brinkman_porous_channel_closed_form(dp):
    # Eq. 1 / Eq. 3 in the same channel filled with porosity d (reading 3).
    # With tau = 1 the collision returns f^eq(rho, d u), so for a fully
    # developed flow u(y) e_x the moments after streaming give, to first order
    # in u and in the pressure gradient, the discrete Brinkman balance
    #   d nu (u(y+1) - 2 u(y) + u(y-1)) - (1 - d) u(y) = (1/rho) dp/dx = G,
    # whose solution with u(0) = u(H) = 0 is
    #   u = (G/beta) (cosh(k (y - H/2)) / cosh(k H/2) - 1),
    #   beta = 1 - d,  2 (cosh k - 1) = beta / (d nu).
    prof, G, P = _channel_steady(dp)
    H = P.dims[1]
    y = np.arange(H)
    beta = (1.0 - dp) / P.tau0
    k = math.acosh(1.0 + beta / (2.0 * dp * P.nu0))
    shape = np.cosh(k * (y - H / 2)) / math.cosh(k * H / 2) - 1.0
    shape[0] = 0.0
    A = (prof * shape).sum() / (shape ** 2).sum()
    assert np.abs(prof - A * shape).max() <= 1e-4 * np.abs(A * shape).max()
    assert abs(A / (G / beta) - 1.0) <= 1e-3


def test_parabolic_inflow_profile_channel():
    # the prescribed-profile inflow node (the channel inflow of Sec. 5.1),
    # f = f^eq(1, u_in(y) e_x), in the tau = 1 channel: the inflow column
    # holds the profile, the developed flow carries the same flux through every
    # column and is the Poiseuille profile with -2 nu A = (1/rho) dp/dx.
    # (The equilibrium node fixes rho = 1 while the interior carries the
    # pressure drop, so the flux is below that of the prescribed profile.)
    from oracle import adjoint as adj
    ny, nx = 9, 48
    y = np.arange(ny)
    prof_in = 4 * 0.03 * y * (ny - y) / ny ** 2
    P = Params(9, (nx, ny, 1), tau0=1.0, u_in=0.02, u_in_profile=prof_in[None, :])
    d = np.ones(P.shape)
    d[0, 0, :] = 0.0
    f = hlbm.initial_state(P)
    for _ in range(200):
        f = hlbm.step(f, d, P)
    f, res = adj.newton_steady(f, d, P, iters=12)
    assert res < 1e-13
    rho, u = hlbm.moments(f, P)
    assert np.abs(u[0, 0, :, 0] - prof_in).max() < 1e-15
    flux = (rho[0] * u[0, 0]).sum(axis=0)
    assert np.abs(flux[nx // 3:2 * nx // 3] - flux[nx // 2]).max() <= 1e-5 * flux[nx // 2]
    x0 = nx // 2
    prof = u[0, 0, :, x0].copy()
    prof[0] = 0.0
    para = y * (ny - y)
    A = (prof * para).sum() / (para ** 2).sum()
    assert np.abs(prof - A * para).max() <= 1e-4 * np.abs(A * para).max()
    G = CS2 * (rho[0, 1:, x0 + 5] - rho[0, 1:, x0 - 5]).mean() / 10 / rho[0, 1:, x0].mean()
    assert abs(-2 * P.nu0 * A / G - 1.0) <= 1e-3
