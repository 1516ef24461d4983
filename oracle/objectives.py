"""Objective functionals and their partial derivatives (Sec. 4).

* J_FFA (Sec. 4.2, Eq. obj_ffa): far-field drag over the plane Gamma_J,
  sum rho (u_x u_0 - u_x^2) + sum (p_0 - p), with p = c_s^2 rho and the
  reference pressure p_0 = c_s^2 (rho_0 = 1); unit area weights.
* J_DISS (Sec. 4.3, Eq. obj_diss): sum over Omega_J of
  2 nu S:S + (nu/K) u.u with S = -Pi/(2 tau c_s^2) (the strain from the
  non-equilibrium part, Sec. 4.3) and nu/K = (1 - d)/tau from the porosity
  relation d = 1 - tau nu / K (Sec. 2.1, lattice units).  nu is the
  molecular viscosity, tau in S is the local tau_eff (= tau0 without LES),
  tau in nu/K is tau0.

Readings: the raw velocity u = sum xi f / rho enters both objectives (not
u~); f^neq is taken against f^eq(rho, u~) exactly as the paper defines
f^eq.  Derivatives are written out by the chain rule through rho, u, Pi and
tau_eff and are pinned by central finite differences in the tests.
"""
from __future__ import annotations

import math

import numpy as np

from .hlbm import Params, deq_dut, local_state
from .lattice import CS2

FFA = 1
DISS = 2
MEA = 4


def surface_nodes(d, P: Params):
    """Gamma_s of the momentum-exchange drag (Sec. 4.1) for a smooth porosity
    field.  Reading: the fluid-side boundary nodes of the solid, i.e. cells
    with d >= 1/2 that have a lattice neighbour x + xi_i (inside the domain in
    x, periodic in y and z) with d < 1/2."""
    nz, ny, nx = P.shape
    solid = d < 0.5
    surf = np.zeros_like(solid)
    x = np.arange(nx)
    for i in range(1, P.q):
        cx, cy, cz = (int(c) for c in P.xi[i])
        nb = np.roll(solid, shift=(-cz, -cy), axis=(0, 1))
        xs = x + cx
        ok = (xs >= 0) & (xs < nx)
        shifted = np.zeros_like(solid)
        shifted[..., ok] = nb[..., xs[ok]]
        surf |= shifted
    return surf & ~solid


def mea_value(f, d, P: Params):
    """J_MEA (Sec. 4.1, Eq. obj_mea) with n = e_x, the flow direction:
    (1/A) sum_{x in Gamma_s} sum_i xi_ix (f_i(x + xi_i) - f_ibar(x)), A the
    number of surface nodes (unit lattice area).  Terms whose neighbour
    x + xi_i leaves the domain in x are left out."""
    surf = surface_nodes(d, P)
    A = max(int(surf.sum()), 1)
    nz, ny, nx = P.shape
    x = np.arange(nx)
    total = 0.0
    for i in range(P.q):
        cx, cy, cz = (int(c) for c in P.xi[i])
        if cx == 0:
            continue
        fn = np.roll(f[i], shift=(-cz, -cy), axis=(0, 1))
        xs = x + cx
        ok = (xs >= 0) & (xs < nx)
        term = np.zeros(P.shape)
        term[..., ok] = fn[..., xs[ok]] - f[P.opp[i]][..., ok]
        total += cx * float(term[surf].sum())
    return total / A


def mea_partials(d, P: Params):
    """dJ_MEA/df (constant: J_MEA is linear in f) and dJ_MEA/dd = 0 (the
    surface set is held fixed)."""
    surf = surface_nodes(d, P)
    A = max(int(surf.sum()), 1)
    nz, ny, nx = P.shape
    g = np.zeros((P.q,) + P.shape)
    x = np.arange(nx)
    for i in range(P.q):
        cx, cy, cz = (int(c) for c in P.xi[i])
        if cx == 0:
            continue
        # + xi_ix f_i(y) for y = x + xi_i with x on the surface
        src = np.roll(surf, shift=(cz, cy), axis=(0, 1))
        xs = x - cx
        ok = (xs >= 0) & (xs < nx)
        hit = np.zeros(P.shape, dtype=bool)
        hit[..., ok] = src[..., xs[ok]]
        g[i] += cx * hit / A
        # - xi_ix f_ibar(x) for x on the surface whose neighbour is in the domain
        okx = np.zeros(P.shape, dtype=bool)
        okx[..., (x + cx >= 0) & (x + cx < nx)] = True
        g[P.opp[i]] -= cx * (surf & okx) / A
    return g, np.zeros(P.shape)


def _region_mask(P: Params, objective, regions):
    nz, ny, nx = P.shape
    m = np.zeros((nz, ny, nx), dtype=bool)
    if objective == FFA:
        y0, y1 = regions.ffa_y
        z0, z1 = regions.ffa_z
        m[z0:z1, y0:y1, regions.ffa_x] = True
    else:
        x0, x1, y0, y1, z0, z1 = regions.diss_box
        m[z0:z1, y0:y1, x0:x1] = True
    return m


def cell_values(f, d, P: Params, objective, regions):
    """Per-cell objective density (zero outside the region), shape (nz, ny, nx)."""
    s = local_state(f, d, P)
    mask = _region_mask(P, objective, regions)
    rho, u = s["rho"], s["u"]
    if objective == FFA:
        ux = u[0]
        val = rho * (ux * P.u_in - ux * ux) + (CS2 * 1.0 - CS2 * rho)
    else:
        S = -s["Pi"] / (2.0 * s["tau"] * CS2)
        SS = np.einsum("ab...,ab...->...", S, S)
        val = 2.0 * P.nu0 * SS + (1.0 - d) / P.tau0 * (u * u).sum(axis=0)
    return np.where(mask, val, 0.0)


def value(f, d, P: Params, objective, regions):
    if objective == MEA:
        return mea_value(f, d, P)
    return float(cell_values(f, d, P, objective, regions).sum())


def local_derivatives(f, d, P: Params):
    """Per-cell d feq/d f, d Pi/d f, d Pi/d d for the state f.

    Returns dict with
      dfeq_df (q, q, ...)   d f_i^eq / d f_j
      dfeq_dd (q, ...)      d f_i^eq / d d
      dPi_df  (3, 3, q, ...)
      dPi_dd  (3, 3, ...)
    """
    s = local_state(f, d, P)
    rho, u, ut, feq = s["rho"], s["u"], s["ut"], s["feq"]
    q = P.q
    ext = (1,) * rho.ndim
    G = deq_dut(rho, ut, P)                              # (q, 3, ...)
    # d rho/d f_j = 1;  d u_a/d f_j = (xi_ja - u_a)/rho;  d u~_a/d f_j = d * that
    du_df = (P.xif.T.reshape((3, q) + ext) - u[:, None]) / rho     # (3, q, ...)
    dut_df = d * du_df
    dfeq_df = (feq / rho)[:, None] + np.einsum("ia...,aj...->ij...", G, dut_df)
    us = np.asarray(P.u_s, dtype=np.float64).reshape((3,) + ext)
    v = u - us                                           # d u~/d d
    dfeq_dd = np.einsum("ia...,a...->i...", G, v)
    eye = np.einsum("ja,jb->abj", P.xif, P.xif).reshape((3, 3, q) + ext)
    dPi_df = eye - np.einsum("ia,ib,ij...->abj...", P.xif, P.xif, dfeq_df)
    dPi_dd = -np.einsum("ia,ib,i...->ab...", P.xif, P.xif, dfeq_dd)
    return dict(state=s, dfeq_df=dfeq_df, dfeq_dd=dfeq_dd, dPi_df=dPi_df,
                dPi_dd=dPi_dd, du_df=du_df)


def _dnorm(s, dPi):
    norm = s["norm"]
    safe = np.where(norm > 1e-30, norm, 1.0)
    g = np.einsum("ab...,ab...->...", s["Pi"], dPi)
    return np.where(norm > 1e-30, g / safe, 0.0)


def tau_derivative(s, P: Params, dPi, tau_base):
    """d tau_eff for a perturbation dPi of Pi (zero when C_S = 0)."""
    if P.Cs == 0.0:
        return np.zeros(s["norm"].shape)
    c = (P.Cs ** 2 / CS2) * math.sqrt(2.0) / (2.0 * CS2)
    dn = _dnorm(s, dPi)
    return c * dn / (2.0 * s["tau"] - tau_base)


def partials(f, d, P: Params, objective, regions):
    """(dJ/df (q, nz, ny, nx), dJ/dd (nz, ny, nx)) of the instantaneous objective."""
    if objective == MEA:
        return mea_partials(d, P)
    L = local_derivatives(f, d, P)
    s = L["state"]
    mask = _region_mask(P, objective, regions)
    rho, u = s["rho"], s["u"]
    q = P.q
    if objective == FFA:
        # J = m_x u0 - m_x^2/rho + c_s^2 - c_s^2 rho with m = rho u
        dJ_drho = u[0] * u[0] - CS2
        dJ_dmx = P.u_in - 2.0 * u[0]
        dJdf = dJ_drho[None] + P.xif[:, 0].reshape((q,) + (1,) * rho.ndim) * dJ_dmx[None]
        dJdd = np.zeros_like(rho)
    else:
        tau = s["tau"]
        Pi = s["Pi"]
        PP = np.einsum("ab...,ab...->...", Pi, Pi)
        # J1 = 2 nu S:S = 2 nu * PP / (4 tau^2 c_s^4)
        k = 2.0 * P.nu0 / (4.0 * CS2 * CS2)
        dPP_df = 2.0 * np.einsum("ab...,abj...->j...", Pi, L["dPi_df"])
        dtau_df = np.stack([tau_derivative(s, P, L["dPi_df"][:, :, j], P.tau0) for j in range(q)])
        dJ1_df = k * (dPP_df / tau ** 2 - 2.0 * PP * dtau_df / tau ** 3)
        # J2 = (1-d)/tau0 * u.u
        dJ2_df = (1.0 - d) / P.tau0 * 2.0 * np.einsum("a...,aj...->j...", u, L["du_df"])
        dJdf = dJ1_df + dJ2_df
        dPP_dd = 2.0 * np.einsum("ab...,ab...->...", Pi, L["dPi_dd"])
        dtau_dd = tau_derivative(s, P, L["dPi_dd"], P.tau0)
        dJdd = k * (dPP_dd / tau ** 2 - 2.0 * PP * dtau_dd / tau ** 3) - (u * u).sum(axis=0) / P.tau0
    return np.where(mask[None], dJdf, 0.0), np.where(mask, dJdd, 0.0)


def porous_drag_force(f, d, P: Params, body):
    """x-force of the fluid on a porous body (Sec. 5.1, the F_x of
    c_D = 2 F_x / (rho u^2 D)).  Reading: the force is the momentum the
    collision removes from the fluid in the body's cells per step,
    F_x = -sum_{x in body} sum_i xi_ix (C(f)_i - f_i), which for the porous
    equilibrium is the Brinkman force density (1 - d) rho (u_x - u_s,x) / tau_eff
    summed over the body (Sec. 2.1; the collision invariant pinned in the
    tests).  ``body`` is a boolean mask of shape (nz, ny, nx)."""
    from .hlbm import collide
    fs, _ = collide(f, d, P)
    dm = np.tensordot(P.xif[:, 0], fs - f, axes=(0, 0))     # (nz, ny, nx)
    return -float(dm[body].sum())
