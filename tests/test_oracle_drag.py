"""The oracle's primal against the drag the paper prints for its primal
validation (Sec. 5.1): the 2D Schaefer-Turek cylinder at Re = 20 with the
cylinder as an HLBM porous body (d = 0 inside, d = 1 in the fluid),
reference c_D* = 5.58, and the paper's own HLBM errors at N = 20, 40, 80
cells per diameter (tests/golden/sec5_1_schaefer_turek_drag.txt).

The steady state is reached by Newton steps with the oracle's exact step
Jacobian (``adjoint.newton_steady``, residual below 1e-12), from a few
hundred time steps.  Geometry: channel of height 4.1 D and length 22 D, one
solid row (d = 0) as the wall of the y-periodic domain, parabolic inflow
through the prescribed-profile inflow node, cylinder centred 2 D from the
inflow and the wall.  The equilibrium inflow node holds rho = 1, so the
flow rate it delivers falls short of the prescribed one; the profile is
rescaled once to the measured mean velocity (Re = u_mean D / nu).

Why not self-convergence on the 200 x 80 cylinder case: its tanh blending
has a width fixed in cells (2), so the body's effective diameter changes
with D (the oracle gives c_D = 11.4 at D = 10 and 5.9 at D = 20 there); a
resolution study on it measures the interface model, not the scheme.
"""
import os

import numpy as np

from oracle import adjoint as adj
from oracle import hlbm
from oracle import objectives as obj


def _golden():
    path = os.path.join(os.path.dirname(__file__), "golden", "sec5_1_schaefer_turek_drag.txt")
    ref, errs = None, {}
    for line in open(path):
        parts = line.split()
        if not parts or parts[0].startswith("#"):
            continue
        if parts[0] == "cd_reference":
            ref = float(parts[1])
        elif parts[0] == "hlbm_error":
            errs[int(parts[1])] = float(parts[2])
    return ref, errs


def _schaefer_turek_cd(N, tau, pre_steps):
    ny, nx = int(round(4.1 * N)), 22 * N
    y, x = np.mgrid[0:ny, 0:nx]
    body = (x - 2.0 * N) ** 2 + (y - 2.0 * N) ** 2 < (N / 2.0) ** 2
    d = np.ones((1, ny, nx))
    d[0][body] = 0.0
    d[0, 0, :] = 0.0
    nu = (tau - 0.5) / 3.0
    u_target = 20.0 * nu / N
    yy = np.arange(ny, dtype=np.float64)
    shape = 4.0 * yy * (ny - yy) / ny ** 2
    u_max = 1.5 * u_target
    f = None
    for _ in range(2):
        P = hlbm.Params(9, (nx, ny, 1), tau0=tau, u_in=u_target,
                        u_in_profile=(u_max * shape)[None, :])
        if f is None:
            f = hlbm.initial_state(P)
            for _ in range(pre_steps):
                f = hlbm.step(f, d, P)
        f, res = adj.newton_steady(f, d, P, iters=12, tol=1e-12)
        assert res < 1e-12
        rho, u = hlbm.moments(f, P)
        u_mean = float((rho[0, 1:, N] * u[0, 0, 1:, N]).sum() / ny)
        u_max *= u_target / u_mean
    F = obj.porous_drag_force(f, d, P, body[None])
    # the same force from the Brinkman density (1 - d) rho u_x / tau over the body
    F2 = float(((1.0 - d) * rho * u[0])[body[None]].sum() / tau)
    assert abs(F - F2) <= 1e-12 * abs(F)
    return 2.0 * F / (u_mean ** 2 * N), u_mean * N / nu


def test_schaefer_turek_drag_within_the_papers_hlbm_error_band():
    ref, paper_err = _golden()
    cd10, re10 = _schaefer_turek_cd(10, 0.8, 400)
    cd20, re20 = _schaefer_turek_cd(20, 1.0, 800)
    for re in (re10, re20):
        assert abs(re - 20.0) < 0.2
    e10 = abs(cd10 - ref) / ref
    e20 = abs(cd20 - ref) / ref
    # second-order HLBM (the paper: 3.07 % at N = 20) gives about 4x that at N = 10;
    # here the Mach number also differs between the two (0.52 at both, by tau)
    assert e20 <= 2.0 * paper_err[20]
    assert e10 <= 4.0 * paper_err[20] * 1.5
    assert e20 < e10
