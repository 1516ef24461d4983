"""Primal HLBM in FP64: moments, porous equilibrium, Smagorinsky tau_eff,
BGK collision, the third-order recursive regularised collision of the
turbulent model (Sec. 2.2, Eq. HRRLBM), streaming and the inflow/outflow
nodes.

State layout: ``f`` has shape (q, nz, ny, nx); x is the fastest axis and
nz = 1 in 2D.  A 'canonical state' f^n is the post-streaming,
post-boundary, pre-collision population field at step n; moments,
objectives and averages are taken there.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Tuple

import numpy as np

from .lattice import CS2, velocity_set


@dataclasses.dataclass
class Params:
    """Physical and lattice parameters of one case (lattice units)."""

    q: int
    dims: Tuple[int, int, int]          # (nx, ny, nz)
    tau0: float                         # molecular relaxation time
    Cs: float = 0.0                     # Smagorinsky constant (0: plain BGK)
    u_in: float = 0.05                  # inflow velocity
    u_s: Tuple[float, float, float] = (0.0, 0.0, 0.0)  # solid velocity
    collision: str = "bgk"              # "bgk" (Eq. 2) or "rr" (Eq. HRRLBM)
    u_in_profile: Optional[np.ndarray] = None  # (nz, ny) inflow u_x per row; None: uniform u_in

    def __post_init__(self):
        if self.collision not in ("bgk", "rr"):
            raise ValueError("collision must be 'bgk' or 'rr'")
        self.xi, self.w, self.opp = velocity_set(self.q)
        self.xif = self.xi.astype(np.float64)
        self.H2, self.H3 = hermite_tensors(self.xif, 2 if self.q == 9 else 3)

    @property
    def shape(self):
        nx, ny, nz = self.dims
        return (nz, ny, nx)

    @property
    def nu0(self):
        # nu = c_s^2 (tau - 1/2)   (Sec. 2.1, viscosity-relaxation relation)
        return CS2 * (self.tau0 - 0.5)


def hermite_tensors(xi, dim):
    """Hermite polynomials of the discrete velocities (Sec. 2.2):
    H2_ab = xi_a xi_b - c_s^2 delta_ab, shape (q, 3, 3);
    H3_abc = xi_a xi_b xi_c - c_s^2 (xi_a delta_bc + xi_b delta_ac + xi_c delta_ab),
    shape (q, 3, 3, 3).  Indices run over the lattice's ``dim`` axes (the
    z entries are zero in 2D)."""
    I = np.diag([1.0, 1.0, 1.0 if dim == 3 else 0.0])
    H2 = np.einsum("ia,ib->iab", xi, xi) - CS2 * I[None]
    H3 = (np.einsum("ia,ib,ic->iabc", xi, xi, xi)
          - CS2 * (np.einsum("ia,bc->iabc", xi, I) + np.einsum("ib,ac->iabc", xi, I)
                   + np.einsum("ic,ab->iabc", xi, I)))
    return H2, H3


def tau_from_reynolds(u0: float, L: float, Re: float) -> float:
    """tau = nu / c_s^2 + 1/2 with nu = u0 L / Re (Sec. 2.1 and Sec. 5.2)."""
    return (u0 * L / Re) / CS2 + 0.5


# ---------------------------------------------------------------------------
# local (per-cell) quantities; arrays carry the cell axes after the first
# ---------------------------------------------------------------------------

def moments(f, P: Params):
    """rho = sum_i f_i, u = (1/rho) sum_i xi_i f_i  (Sec. 2.1, Eq. 4-5)."""
    rho = f.sum(axis=0)
    m = np.tensordot(P.xif.T, f, axes=(1, 0))     # (3, ...)
    return rho, m / rho


def porous_velocity(u, d, P: Params):
    """u~ = d u + (1 - d) u_s: the HLBM modified velocity (Sec. 2.1, after Eq. 3).

    The paper writes u~ = d u, i.e. a solid at rest; u_s generalises it to a
    moving solid and defaults to 0."""
    us = np.asarray(P.u_s, dtype=np.float64).reshape((3,) + (1,) * (u.ndim - 1))
    return d * u + (1.0 - d) * us


def equilibrium(rho, ut, P: Params):
    """Second-order equilibrium f_i^eq(rho, u~) (Sec. 2.1, Eq. 3)."""
    cu = np.tensordot(P.xif, ut, axes=(1, 0))       # (q, ...)
    uu = (ut * ut).sum(axis=0)
    wexp = P.w.reshape((P.q,) + (1,) * rho.ndim)
    return wexp * rho * (1.0 + cu / CS2 + cu * cu / (2 * CS2 * CS2) - uu / (2 * CS2))


def deq_dut(rho, ut, P: Params):
    """d f_i^eq / d u~_a, shape (q, 3, ...)."""
    cu = np.tensordot(P.xif, ut, axes=(1, 0))        # (q, ...)
    q = P.q
    ext = (1,) * rho.ndim
    xi = P.xif.reshape((q, 3) + ext)
    wexp = P.w.reshape((q, 1) + ext)
    return wexp * rho * (xi / CS2 + cu[:, None] * xi / (CS2 * CS2) - ut[None] / CS2)


def noneq_stress(f, feq, P: Params):
    """Pi_ab = sum_i xi_ia xi_ib (f_i - f_i^eq), shape (3, 3, ...) (Sec. 4.3, Eq. for S)."""
    return np.einsum("ia,ib,i...->ab...", P.xif, P.xif, f - feq)


def tau_effective(Pi, tau_base, P: Params):
    """Local relaxation time with the Smagorinsky eddy viscosity (Sec. 2.2).

    tau_eff = (nu_mo + nu_turb)/c_s^2 + 1/2 with nu_turb = (C_S)^2 |S| and
    S = -Pi / (2 tau_eff c_s^2), |S| = sqrt(2 S:S).  Since S itself depends
    on tau_eff, tau_eff solves
        tau_eff^2 - tau_base tau_eff - (C_S^2 / c_s^2) * sqrt(2) ||Pi|| / (2 c_s^2) = 0,
    of which the positive root is taken.  With C_S = 0 this is tau_base.
    """
    norm = np.sqrt(np.einsum("ab...,ab...->...", Pi, Pi))
    if P.Cs == 0.0:
        return np.full(norm.shape, float(tau_base)), norm
    return tau_of_norm(norm, tau_base, P), norm


def tau_of_norm(norm, tau_base, P: Params):
    """The positive root above as a function of ||Pi|| (also for complex input)."""
    c = (P.Cs ** 2 / CS2) * math.sqrt(2.0) / (2.0 * CS2)   # = 9 sqrt(2)/2 * Cs^2
    return 0.5 * (tau_base + np.sqrt(tau_base * tau_base + 4.0 * c * norm))


def local_state(f, d, P: Params, tau_base=None):
    """All per-cell quantities of the collision at state f."""
    if tau_base is None:
        tau_base = P.tau0
    rho, u = moments(f, P)
    ut = porous_velocity(u, d, P)
    feq = equilibrium(rho, ut, P)
    Pi = noneq_stress(f, feq, P)
    te, norm = tau_effective(Pi, tau_base, P)
    return dict(rho=rho, u=u, ut=ut, feq=feq, Pi=Pi, tau=te, norm=norm)


def equilibrium3(rho, ut, P: Params):
    """Third-order Hermite equilibrium of the recursive regularised model
    (Sec. 2.2): w_i (a0^(0) + H1_i.a0^(1)/c_s^2 + H2_i:a0^(2)/(2 c_s^4)
    + H3_i:a0^(3)/(6 c_s^6)) with a0^(0) = rho and a0^(n) = a0^(n-1) u~,
    ':' the full tensor contraction."""
    a1 = rho * ut
    a2 = np.einsum("a...,b...->ab...", a1, ut)
    a3 = np.einsum("ab...,c...->abc...", a2, ut)
    h1 = np.tensordot(P.xif, a1, axes=(1, 0))
    h2 = np.tensordot(P.H2, a2, axes=([1, 2], [0, 1]))
    h3 = np.tensordot(P.H3, a3, axes=([1, 2, 3], [0, 1, 2]))
    wexp = P.w.reshape((P.q,) + (1,) * rho.ndim)
    return wexp * (rho[None] + h1 / CS2 + h2 / (2 * CS2 ** 2) + h3 / (6 * CS2 ** 3))


def regularised_noneq(fneq, ut, P: Params):
    """f^(1) of Sec. 2.2: the non-equilibrium part expanded in Hermite
    polynomials up to third order.  Reading: a1^(n) = sum_i H_i^(n) f^neq_i
    for n <= 2 (f^neq = f - f^eq), and the third-order coefficient is built
    recursively, a1^(3)_abc = u~_a a1^(2)_bc + u~_b a1^(2)_ac + u~_c a1^(2)_ab,
    as in the recursive regularised schemes the paper builds on."""
    a0 = fneq.sum(axis=0)
    a1 = np.tensordot(P.xif.T, fneq, axes=(1, 0))
    a2 = np.tensordot(P.H2.transpose(1, 2, 0), fneq, axes=(2, 0))
    a3 = (np.einsum("a...,bc...->abc...", ut, a2) + np.einsum("b...,ac...->abc...", ut, a2)
          + np.einsum("c...,ab...->abc...", ut, a2))
    h1 = np.tensordot(P.xif, a1, axes=(1, 0))
    h2 = np.tensordot(P.H2, a2, axes=([1, 2], [0, 1]))
    h3 = np.tensordot(P.H3, a3, axes=([1, 2, 3], [0, 1, 2]))
    wexp = P.w.reshape((P.q,) + (1,) * a0.ndim)
    return wexp * (a0[None] + h1 / CS2 + h2 / (2 * CS2 ** 2) + h3 / (6 * CS2 ** 3))


def collide_rr(f, d, P: Params, tau=None, tau_base=None):
    """Recursive regularised collision f* = f^eq + (1 - 1/tau_eff) f^(1)
    (Sec. 2.2, Eq. HRRLBM) with the third-order porous equilibrium at
    (rho, u~).  tau_eff is the Smagorinsky relaxation time of the
    non-equilibrium stress (Eq. tauEff; unchanged from the BGK model, since
    the third-order terms do not alter second moments), or the given
    ``tau`` (frozen)."""
    if tau_base is None:
        tau_base = P.tau0
    rho, u = moments(f, P)
    ut = porous_velocity(u, d, P)
    feq = equilibrium3(rho, ut, P)
    fneq = f - feq
    if tau is None:
        tau, _ = tau_effective(noneq_stress(f, feq, P), tau_base, P)
    f1 = regularised_noneq(fneq, ut, P)
    return feq + (1.0 - 1.0 / tau) * f1


def collide(f, d, P: Params):
    """One collision: BGK relaxation f* = f - (f - f^eq)/tau_eff (Sec. 2.1,
    Eq. 2), or the recursive regularised collision when P.collision = "rr"."""
    s = local_state(f, d, P)
    if P.collision == "rr":
        return collide_rr(f, d, P, tau=s["tau"]), s
    return f - (f - s["feq"]) / s["tau"], s


# ---------------------------------------------------------------------------
# streaming and boundary nodes
# ---------------------------------------------------------------------------

def stream(fs, P: Params):
    """f_i(x + xi_i) = f*_i(x): periodic in y and z; populations leaving the
    domain through x = 0 or x = nx-1 are dropped and nothing enters there
    (those columns are boundary nodes that the next call overwrites)."""
    out = np.empty_like(fs)
    for i in range(P.q):
        cx, cy, cz = (int(c) for c in P.xi[i])
        a = np.roll(fs[i], shift=(cz, cy, cx), axis=(0, 1, 2))
        if cx == 1:
            a[..., 0] = 0.0
        elif cx == -1:
            a[..., -1] = 0.0
        out[i] = a
    return out


def inflow_state(P: Params, shape=None):
    """Equilibrium at rho = 1 and u = (u_in, 0, 0) (inflow Dirichlet node)."""
    if shape is None:
        shape = ()
    rho = np.ones(shape)
    u = np.zeros((3,) + tuple(shape))
    u[0] = P.u_in
    return equilibrium(rho, u, P)


def apply_boundary(f, P: Params):
    """Inflow column x = 0: f = f^eq(1, u_in e_x).  Outflow column x = nx-1:
    f = f^eq(1, u(x = nx-2)) -- a constant-pressure outlet with the velocity
    copied from the neighbouring column.  The paper states a velocity
    inflow, a pressure outflow and periodic lateral walls (Sec. 5.2.1) but
    not the discrete scheme; these equilibrium nodes are the reading used
    throughout."""
    f = f.copy()
    nz, ny, nx = P.shape
    if P.u_in_profile is None:
        f[..., 0] = inflow_state(P, (nz, ny))
    else:
        # a prescribed velocity profile (e.g. the parabolic channel inflow of
        # the Schaefer-Turek benchmark, Sec. 5.1)
        u = np.zeros((3, nz, ny))
        u[0] = P.u_in_profile
        f[..., 0] = equilibrium(np.ones((nz, ny)), u, P)
    rho, u = moments(f[..., nx - 2], P)
    f[..., nx - 1] = equilibrium(np.ones_like(rho), u, P)
    return f


def step(f, d, P: Params):
    """One time step Phi(f) = B(S(C(f))) from canonical state to canonical state."""
    fs, _ = collide(f, d, P)
    return apply_boundary(stream(fs, P), P)


def initial_state(P: Params, u_perturb=None):
    """f^0 = f^eq(1, u_in e_x + u_perturb) everywhere, then boundary nodes."""
    nz, ny, nx = P.shape
    u = np.zeros((3, nz, ny, nx))
    u[0] = P.u_in
    if u_perturb is not None:
        u = u + u_perturb
    f = equilibrium(np.ones((nz, ny, nx)), u, P)
    return apply_boundary(f, P)


def macroscopic(f, P: Params):
    rho, u = moments(f, P)
    return rho, u
