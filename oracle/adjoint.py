"""Linearised step, (mean-flow) adjoint iteration and gradient in FP64.

One primal step is Phi(f; d) = B(S(C(f; d))) (collision C, streaming S,
boundary nodes B; see ``hlbm.step``).  The adjoint equations of the paper
(Eq. adjoint_steady, Eq. adjoint_unsteady) iterate, in the sign convention
used here,

    lambda^{k+1} = A^T lambda^k + g_bar,     A = dPhi/df at f_bar,

with g_bar the (time-averaged) dJ/df, until the update is below a tolerance
(Algorithm 1).  The fixed point solves (I - A^T) lambda = g_bar.  The
gradient (Eq. gradients_steady, Eq. gradients_unsteady) is

    dJ/dd = dJ/dd_bar + (dPhi/dd)^T lambda,
    (dPhi/dd)^T lambda = sum_i mu_i dC_i/dd,   mu = S^T B_f^T lambda.

The paper's adjoint variable carries the opposite sign (phi = -mu shifted
by one step); the gradient does not depend on that convention.

Linearisation modes (Sec. 5.4):
* EXACT: the full Jacobian of the collision at f_bar, including the
  derivative of the Smagorinsky tau_eff (the extra source term of the
  differentiated LES collision).
* FTA (frozen turbulence): tau_eff is frozen at tau_base + the time
  average of tau_eff - tau0; its derivatives are dropped.
With C_S = 0 both are the plain BGK Jacobian.  ``tau_adj`` (Sec. 5.4, the
adjoint regularisation) replaces tau0 as tau_base in the linearised
operator only.

The Jacobians are assembled as scipy.sparse matrices from per-cell dense
q x q blocks written out by the chain rule; tests pin them against central
differences of ``hlbm.step``.  For the recursive regularised collision
(Sec. 2.2) the blocks are taken by complex-step differentiation of
``hlbm.collide_rr`` (Squire and Trapp, 1998: f'(x) = Im f(x + i h)/h, exact
to rounding for tiny h since nothing is subtracted), with the same
EXACT / FTA / tau_adj semantics.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import objectives as obj
from .hlbm import Params, deq_dut, local_state, moments, step

EXACT = 0
FTA = 1


def cell_index(P: Params):
    nx, ny, nz = P.dims
    return np.arange(nx * ny * nz).reshape(nz, ny, nx)


CSTEP = 1e-30


def _rr_complex(fc, dc, P: Params, mode, tau_base, tau_t_bar):
    """collide_rr on complex inputs with the relaxation time of ``mode``."""
    from .hlbm import collide_rr, equilibrium3, noneq_stress, porous_velocity, tau_of_norm
    if P.Cs > 0.0 and mode == FTA:
        tau = tau_base + tau_t_bar
    elif P.Cs > 0.0:
        rho, u = moments(fc, P)
        Pi = noneq_stress(fc, equilibrium3(rho, porous_velocity(u, dc, P), P), P)
        n2 = np.einsum("ab...,ab...->...", Pi, Pi)
        # |Pi| -> 0: the derivative of |Pi| is taken as 0 there (as for BGK)
        small = n2.real <= 1e-60
        norm = np.where(small, 0.0, np.sqrt(np.where(small, 1.0, n2)))
        tau = tau_of_norm(norm, tau_base, P)
    else:
        tau = np.full(P.shape, float(tau_base))
    return collide_rr(fc, dc, P, tau=tau)


def rr_collision_jacobians(f, d, P: Params, mode=EXACT, tau_adj=None, tau_t_bar=None):
    """dC_i/df_j and dC_i/dd of the recursive regularised collision by complex
    steps: perturbing f_j (or d) in every cell at once gives column j of
    every cell's block, the collision being local."""
    tau_base = P.tau0 if tau_adj is None else float(tau_adj)
    if P.Cs > 0.0 and mode == FTA and tau_t_bar is None:
        raise ValueError("FTA needs the averaged turbulent relaxation time")
    q = P.q
    JC = np.empty((q, q) + P.shape)
    for j in range(q):
        fc = f.astype(np.complex128)
        fc[j] += 1j * CSTEP
        JC[:, j] = _rr_complex(fc, d.astype(np.complex128), P, mode, tau_base, tau_t_bar).imag / CSTEP
    dc = d + 1j * CSTEP
    Cd = _rr_complex(f.astype(np.complex128), dc, P, mode, tau_base, tau_t_bar).imag / CSTEP
    return JC, Cd


def collision_jacobians(f, d, P: Params, mode=EXACT, tau_adj=None, tau_t_bar=None):
    """Per-cell dC_i/df_j (q, q, nz, ny, nx) and dC_i/dd (q, nz, ny, nx) at f."""
    if P.collision == "rr":
        return rr_collision_jacobians(f, d, P, mode, tau_adj, tau_t_bar)
    tau_base = P.tau0 if tau_adj is None else float(tau_adj)
    L = obj.local_derivatives(f, d, P)
    s = local_state(f, d, P, tau_base)
    q = P.q
    if P.Cs > 0.0 and mode == FTA:
        if tau_t_bar is None:
            raise ValueError("FTA needs the averaged turbulent relaxation time")
        tau = tau_base + tau_t_bar
    else:
        tau = s["tau"]
    om = 1.0 / tau
    feq = s["feq"]
    eye = np.eye(q).reshape((q, q) + (1,) * om.ndim)
    JC = (1.0 - om) * eye + om * L["dfeq_df"]
    Cd = om * L["dfeq_dd"]
    if P.Cs > 0.0 and mode == EXACT:
        # C_i = (1 - om) f_i + om feq_i  =>  + (feq_i - f_i) d om ;  d om = -om^2 d tau
        dtau_df = np.stack([obj.tau_derivative(s, P, L["dPi_df"][:, :, j], tau_base)
                            for j in range(q)])
        dom_df = -om * om * dtau_df
        JC = JC + (feq - f)[:, None] * dom_df[None, :]
        dtau_dd = obj.tau_derivative(s, P, L["dPi_dd"], tau_base)
        Cd = Cd + (feq - f) * (-om * om * dtau_dd)
    return JC, Cd


def outlet_jacobian(f, P: Params):
    """d f_i(x = nx-1) / d f_j(x = nx-2) of the outflow node, (q, q, nz, ny)."""
    nz, ny, nx = P.shape
    rho, u = moments(f[..., nx - 2], P)
    G = deq_dut(np.ones_like(rho), u, P)                    # (q, 3, nz, ny)
    du_df = (P.xif.T.reshape((3, P.q, 1, 1)) - u[:, None]) / rho
    return np.einsum("ia...,aj...->ij...", G, du_df)


def streaming_matrix(P: Params):
    """S as a sparse permutation-like matrix on index i*N + cell."""
    nz, ny, nx = P.shape
    N = nx * ny * nz
    idx = cell_index(P)
    rows, cols = [], []
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    for i in range(P.q):
        cx, cy, cz = (int(c) for c in P.xi[i])
        xd = x + cx
        ok = (xd >= 0) & (xd < nx)
        dest = idx[(z + cz) % nz, (y + cy) % ny, np.clip(xd, 0, nx - 1)]
        rows.append(i * N + dest[ok])
        cols.append(i * N + idx[ok])
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    return sp.csr_matrix((np.ones(rows.size), (rows, cols)), shape=(P.q * N, P.q * N))


def boundary_matrix(f_streamed, P: Params):
    """B_f: identity on interior columns, zero rows on the inflow column,
    the outflow rows coupled to column nx-2 through ``outlet_jacobian``."""
    nz, ny, nx = P.shape
    N = nx * ny * nz
    idx = cell_index(P)
    q = P.q
    keep = np.ones((nz, ny, nx), dtype=bool)
    keep[..., 0] = False
    keep[..., nx - 1] = False
    rows = [i * N + idx[keep] for i in range(q)]
    cols = list(rows)
    vals = [np.ones(int(keep.sum()))] * q
    Jo = outlet_jacobian(f_streamed, P)
    for i in range(q):
        for j in range(q):
            rows.append(i * N + idx[..., nx - 1].ravel())
            cols.append(j * N + idx[..., nx - 2].ravel())
            vals.append(Jo[i, j].ravel())
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = np.concatenate(vals)
    return sp.csr_matrix((vals, (rows, cols)), shape=(q * N, q * N))


def block_diag_matrix(JC, P: Params):
    nz, ny, nx = P.shape
    N = nx * ny * nz
    q = P.q
    c = np.arange(N)
    rows = (np.arange(q)[:, None, None] * N + c[None, None, :]).repeat(q, axis=1)
    cols = (np.arange(q)[None, :, None] * N + c[None, None, :]).repeat(q, axis=0)
    return sp.csr_matrix((JC.reshape(q, q, N).ravel(), (rows.ravel(), cols.ravel())),
                         shape=(q * N, q * N))


class Linearisation:
    """Step Jacobian A = B_f S C_f and dPhi/dd at the state ``fbar``."""

    def __init__(self, fbar, d, P: Params, mode=EXACT, tau_adj=None, tau_t_bar=None,
                 outlet="canonical", assemble=True):
        """``outlet`` selects the state at which the outflow node is
        linearised: "canonical" uses the velocity of ``fbar`` at x = nx-2
        (the reading used for the mean-flow adjoint and by the CUDA path),
        "streamed" uses S(C(fbar)) there, i.e. the exact derivative of
        ``hlbm.step`` at an arbitrary state.  At a fixed point both agree.

        ``assemble`` = False keeps the collision Jacobian as its per-cell
        q x q blocks and applies A = (B S) C_f factor by factor instead of
        forming the product matrix: the same linear maps for grids where the
        assembled q^2 N-entry matrices would not fit (the direct solve then
        is not available)."""
        from .hlbm import collide, stream
        self.P = P
        nz, ny, nx = P.shape
        self.N = nx * ny * nz
        self.shape = (P.q,) + P.shape
        JC, Cd = collision_jacobians(fbar, d, P, mode, tau_adj, tau_t_bar)
        if outlet == "streamed":
            fs, _ = collide(fbar, d, P)
            Bm = boundary_matrix(stream(fs, P), P)
        else:
            Bm = boundary_matrix(fbar, P)
        Sm = streaming_matrix(P)
        self.BS = (Bm @ Sm).tocsr()
        self.BST = self.BS.T.tocsr()
        self.assembled = assemble
        if not assemble:
            self.JC, self.Cd = JC, Cd
            return
        self.A = (self.BS @ block_diag_matrix(JC, P)).tocsr()
        N = self.N
        cells = np.arange(N)
        Cdm = sp.csr_matrix((Cd.reshape(P.q, N).ravel(),
                             ((np.arange(P.q)[:, None] * N + cells[None]).ravel(),
                              np.tile(cells, P.q))), shape=(P.q * N, N))
        self.D = (self.BS @ Cdm).tocsr()
        self.AT = self.A.T.tocsr()
        self.DT = self.D.T.tocsr()

    def jvp(self, v):
        """A v (tangent of one step), v shaped like f."""
        if not self.assembled:
            cv = np.einsum("ij...,j...->i...", self.JC, v.reshape(self.shape))
            return (self.BS @ cv.ravel()).reshape(v.shape)
        return (self.A @ v.ravel()).reshape(v.shape)

    def vjp(self, lam):
        """A^T lam, shaped like f."""
        if not self.assembled:
            m = (self.BST @ lam.ravel()).reshape(self.shape)
            return np.einsum("ij...,i...->j...", self.JC, m).reshape(lam.shape)
        return (self.AT @ lam.ravel()).reshape(lam.shape)

    def mu(self, lam):
        """mu = S^T B_f^T lam: the adjoint pulled back through stream and boundary."""
        return (self.BST @ lam.ravel()).reshape(lam.shape)

    def dd_vjp(self, lam):
        """(dPhi/dd)^T lam, one value per cell, shape (nz, ny, nx)."""
        if not self.assembled:
            return (self.mu(lam.reshape(self.shape)) * self.Cd).sum(axis=0)
        return (self.DT @ lam.ravel()).reshape(self.P.shape)


def solve_adjoint(lin: Linearisation, gbar, tol=1e-10, max_iter=100000, lam0=None):
    """Iterate lambda <- A^T lambda + g_bar from lambda = 0 until
    ||lambda^{k+1} - lambda^k||_2 / ||g_bar||_2 <= tol (Algorithm 1).
    Returns (lambda, iterations, final residual)."""
    g = gbar.ravel()
    gn = float(np.sqrt(np.dot(g, g)))
    lam = np.zeros_like(g) if lam0 is None else lam0.ravel().copy()
    r = np.inf
    for k in range(1, max_iter + 1):
        new = lin.vjp(lam) + g
        diff = new - lam
        r = float(np.sqrt(np.dot(diff, diff))) / (gn if gn > 0 else 1.0)
        lam = new
        if r <= tol:
            return lam.reshape(gbar.shape), k, r
    return lam.reshape(gbar.shape), max_iter, r


def solve_adjoint_direct(lin: Linearisation, gbar):
    """(I - A^T) lambda = g_bar by a sparse direct solve (small grids)."""
    from scipy.sparse.linalg import spsolve
    n = lin.A.shape[0]
    M = (sp.identity(n, format="csr") - lin.AT).tocsc()
    return spsolve(M, gbar.ravel()).reshape(gbar.shape)


def gradient(lin: Linearisation, lam, dJdd_bar):
    """dJ/dd per cell = dJ/dd_bar + (dPhi/dd)^T lambda, shape (nz, ny, nx)."""
    return dJdd_bar + lin.dd_vjp(lam).reshape(dJdd_bar.shape)


def newton_steady(f, d, P: Params, iters=8, tol=1e-14):
    """Fixed point f = Phi(f) by Newton steps with the exact step Jacobian."""
    from scipy.sparse.linalg import spsolve
    n = f.size
    res = np.inf
    for _ in range(iters):
        r = step(f, d, P) - f
        res = float(np.abs(r).max())
        if res < tol:
            break
        lin = Linearisation(f, d, P, EXACT, outlet="streamed")
        M = (sp.identity(n, format="csr") - lin.A).tocsc()
        f = f + spsolve(M, r.ravel()).reshape(f.shape)
    return f, res


def unsteady_adjoint_gradient(f0, d, P: Params, T: int, objective, regions, checkpoint_every=None):
    """Exact gradient of the short-horizon time average J_T = (1/T) sum_{n<T} J(f^n; d),
    f^{n+1} = Phi(f^n; d) from a fixed f^0, by the discrete unsteady adjoint -- the
    validation reference for the transient sensitivities (App. C), against which the
    mean-flow adjoint is an approximation.

    Backward sweep with the exact step Jacobians at every state:
        lambda^T = 0,  lambda^n = A_n^T lambda^{n+1} + g_n / T   (n = T-1 .. 1),
        dJ_T/dd = (1/T) sum_n dJ/dd(f^n) + sum_{n=0}^{T-2} D_n^T lambda^{n+1},
    A_n = dPhi/df and D_n = dPhi/dd at f^n (outflow node linearised at the streamed
    state: the exact derivative of the step).  The forward states are kept only at
    checkpoints every c = ceil(sqrt(T)) steps and recomputed segment by segment
    during the backward sweep.  Returns (gradient, J_T, forward steps taken)."""
    c = checkpoint_every or int(np.ceil(np.sqrt(T)))
    checkpoints = {}
    f = f0.copy()
    JT = 0.0
    fwd = 0
    for n in range(T):
        if n % c == 0:
            checkpoints[n] = f.copy()
        JT += obj.value(f, d, P, objective, regions) / T
        if n < T - 1:
            f = step(f, d, P)
            fwd += 1
    lam = np.zeros_like(f0)
    G = np.zeros(P.shape)
    for start in sorted(checkpoints, reverse=True):
        end = min(start + c, T)
        seg = [checkpoints[start]]
        for _ in range(start, end - 1):
            seg.append(step(seg[-1], d, P))
            fwd += 1
        for n in range(end - 1, start - 1, -1):
            fn = seg[n - start]
            g, gd = obj.partials(fn, d, P, objective, regions)
            G += gd / T
            lin = Linearisation(fn, d, P, EXACT, outlet="streamed")
            if n < T - 1:
                # lam holds lambda^{n+1}: the step out of f^n carries D_n^T lambda^{n+1}
                G += (lin.DT @ lam.ravel()).reshape(P.shape)
            if n >= 1:
                lam = (lin.AT @ lam.ravel()).reshape(f0.shape) + g / T
    return G, JT, fwd
