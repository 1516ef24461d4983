"""The differentiation form on the Gaussian-random-field design case (D2Q9
400x160, Re 40 on the 60-cell design box, u0 0.05, porosity a seeded Gaussian
random field of correlation length 8 clipped to [0, 1] inside the box,
d = 1 outside; drag J_FFA on the plane x = 300 and dissipation J_DISS over
the whole domain).

* The gradient that ``torch.autograd`` returns through ``HLBMObjective``
  (FP32 populations, steady primal, adjoint to 2e-5, the FP32 floor of its
  update criterion here) against the FP64
  oracle's gradient: the oracle's steady state by Newton steps with its exact
  step Jacobian and its adjoint by a sparse direct solve (Eq. gradients_steady).
  Bound 1e-4 relative L2 over the whole domain.
* The same gradient against central differences of J (h = 1e-4) on 32 seeded
  cells of the design box, J evaluated with FP64 populations (FP32 would
  cancel in the difference) at steady states converged until J changes by
  less than 1e-13 relative between checks.

The oracle runs in a spawned process while the GPU works."""
import concurrent.futures as cf
import multiprocessing as mp

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
H = pytest.importorskip("paper_2606_31707_b300.hlbm")
from paper_2606_31707_b300 import Solver  # noqa: E402
from paper_2606_31707_b300.autograd import HLBMObjective, PrimalSpec  # noqa: E402
from tests.hlbm_cases import oracle_grf_gradients  # noqa: E402
from workloads import Regions, make_workload  # noqa: E402

TOL_ORACLE = 1e-4
# the update criterion of the FP32 fixed-point iteration stalls near 1e-5 on
# this case (the rounding of the FP32 adjoint populations): its tolerance
TOL_ADJ_FP32 = 2e-5
H_FD = 1e-4
N_CELLS = 32


def _regions(wl):
    nx, ny, _ = wl.dims
    r = wl.regions
    return Regions(ffa_x=r.ffa_x, ffa_y=r.ffa_y, ffa_z=r.ffa_z, diss_box=r.diss_box,
                   design_box=(0, nx, 0, ny, 0, 1))


def _tau0(wl):
    return (wl.u0 * wl.L / wl.Re) * 3.0 + 0.5


@pytest.fixture(scope="module")
def oracle_future():
    ex = cf.ProcessPoolExecutor(max_workers=1, mp_context=mp.get_context("spawn"))
    fut = ex.submit(oracle_grf_gradients)
    yield fut
    ex.shutdown(wait=True)


def _steady_J(s, objective, chunk=20000, max_steps=400000):
    """Run the primal from the current state until J changes by < 1e-13 relative."""
    prev = None
    for _ in range(max_steps // chunk):
        s.run_primal(chunk, 1)
        J = s.objective(objective)
        if prev is not None and abs(J - prev) <= 1e-13 * abs(J):
            return J
        prev = J
    raise AssertionError("steady state not reached")


@pytest.mark.parametrize("objective", [H.OBJ_DRAG_FFA, H.OBJ_DISSIPATION])
def test_autograd_grf_gradient_against_oracle_and_central_differences(oracle_future, objective):
    wl = make_workload("grf2d_re40")
    dev = torch.device("cuda", 0)
    R = _regions(wl)
    tau = _tau0(wl)
    # autograd, FP32 populations
    s32 = Solver(9, wl.dims, tau, 0.0, storage=H.FP32, u_in=wl.u0, regions=R)
    spec = PrimalSpec(steps=200000, avg_window=1, objective=objective, tol=TOL_ADJ_FP32,
                      max_iter=1_000_000)
    dt = torch.from_numpy(wl.porosity.astype(np.float32)).to(dev).requires_grad_(True)
    J32 = HLBMObjective.apply(dt, s32, spec)
    J32.backward()
    st, it, res = s32.last_adjoint
    assert st == H.OK and res <= TOL_ADJ_FP32
    G = dt.grad.detach().double().cpu().numpy()
    s32.close()
    # central differences of J with FP64 populations, warm-started at the steady state
    s64 = Solver(9, wl.dims, tau, 0.0, storage=H.FP64, u_in=wl.u0, regions=R)
    s64.set_porosity(wl.porosity)
    J0 = _steady_J(s64, objective)
    f_star = s64.field(H.FIELD_F)
    rng = np.random.default_rng(40)
    x0, x1, y0, y1 = 70, 130, 50, 110
    cells = [(int(rng.integers(y0, y1)), int(rng.integers(x0, x1))) for _ in range(N_CELLS)]
    scale = np.abs(G).max()
    worst = 0.0
    for (y, x) in cells:
        vals = []
        for sgn in (1, -1):
            dp = wl.porosity.copy()
            dp[0, y, x] += sgn * H_FD
            s64.set_porosity(dp)
            s64.set_field(H.FIELD_F, f_star)
            vals.append(_steady_J(s64, objective))
        fd = (vals[0] - vals[1]) / (2 * H_FD)
        worst = max(worst, abs(fd - G[0, y, x]) / scale)
    s64.close()
    assert worst <= 2e-4, worst
    # the FP64 oracle's gradient over the whole domain
    ref = oracle_future.result(timeout=1800)
    assert ref["newton_residual"] < 1e-12
    key = 1 if objective == H.OBJ_DRAG_FFA else 2
    G_ref, J_ref = ref[key]
    rel = float(np.linalg.norm(G - G_ref) / np.linalg.norm(G_ref))
    assert rel <= TOL_ORACLE, rel
    assert abs(J0 - J_ref) <= 1e-10 * abs(J_ref)
    print(f"GRF case objective {objective}: autograd vs oracle rel L2 {rel:.2e}, "
          f"vs central differences {worst:.2e} of max|G|, adjoint {it} sweeps to {res:.1e}")
