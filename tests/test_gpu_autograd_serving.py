"""The differentiation form (torch.autograd.Function porosity -> J) and the
served batched form, on the GPU.

* autograd: gradient against central finite differences of J computed in
  FP64 (h = 1e-4, as for the Gaussian-random-field design case) on seeded
  random cells, and the FP32 gradient against the FP64 one.
* serving: every result is identical alone and in a mix of concurrent
  requests of different sizes, and matches the one-at-a-time path.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
H = pytest.importorskip("paper_2606_31707_b300.hlbm")
from paper_2606_31707_b300 import Solver  # noqa: E402
from paper_2606_31707_b300.autograd import HLBMObjective, PrimalSpec  # noqa: E402
from paper_2606_31707_b300.serve import Request, SensitivityServer, solve_one  # noqa: E402
from workloads import Regions, grf_porosity, serving_porosity  # noqa: E402


def _grf_case(nx=200, ny=80, box=(35, 65, 25, 55)):
    dims = (nx, ny, 1)
    d = grf_porosity(dims, box, corr=4.0, seed=3)
    R = Regions(ffa_x=150, ffa_y=(0, ny), ffa_z=(0, 1), diss_box=(0, nx, 0, ny, 0, 1),
                design_box=(0, nx, 0, ny, 0, 1))
    tau = 0.05 * 30 / 40 / (1 / 3) + 0.5     # Re 40 on the box side, u0 0.05
    return dims, d, R, tau, box


@pytest.mark.parametrize("objective", [H.OBJ_DRAG_FFA, H.OBJ_DISSIPATION])
def test_autograd_gradient_matches_central_fd(objective):
    dims, d, R, tau, box = _grf_case()
    dev = torch.device("cuda", 0)
    s = Solver(9, dims, tau, 0.0, storage=H.FP64, u_in=0.05, regions=R)
    spec = PrimalSpec(steps=40000, avg_window=1, objective=objective, tol=1e-12, max_iter=400000)
    dt = torch.from_numpy(d).to(dev).requires_grad_(True)
    J = HLBMObjective.apply(dt, s, spec)
    J.backward()
    G = dt.grad.detach().cpu().numpy()
    # central differences (h = 1e-4) warm-started from the steady state
    f_star = s.field(H.FIELD_F)
    spec_fd = PrimalSpec(steps=20000, avg_window=1, objective=objective, warm_start=True)
    rng = np.random.default_rng(11)
    cells = [(int(rng.integers(box[2], box[3])), int(rng.integers(box[0], box[1]))) for _ in range(8)]
    h = 1e-4
    for (y, x) in cells:
        vals = []
        for sgn in (1, -1):
            dp = d.copy()
            dp[0, y, x] += sgn * h
            s.set_field(H.FIELD_F, f_star)
            with torch.no_grad():
                vals.append(HLBMObjective.apply(torch.from_numpy(dp).to(dev), s, spec_fd).item())
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - G[0, y, x]) <= 1e-5 * np.abs(G).max() + 1e-6 * abs(fd), (y, x, fd, G[0, y, x])
    s.close()


def test_autograd_fp32_gradient_within_1e4_of_fp64():
    dims, d, R, tau, box = _grf_case()
    dev = torch.device("cuda", 0)
    Gs = []
    # adjoint tolerances: FP64 1e-11; FP32 1e-5, above the floor of the FP32
    # update criterion
    for storage, tol in ((H.FP64, 1e-11), (H.FP32, 1e-5)):
        s = Solver(9, dims, tau, 0.0, storage=storage, u_in=0.05, regions=R)
        spec = PrimalSpec(steps=40000, avg_window=1, objective=H.OBJ_DISSIPATION, tol=tol,
                          max_iter=1_000_000)
        dt = torch.from_numpy(d.astype(np.float32 if storage == H.FP32 else np.float64)).to(dev)
        dt.requires_grad_(True)
        HLBMObjective.apply(dt, s, spec).backward()
        Gs.append(dt.grad.detach().double().cpu().numpy())
        s.close()
    rel = np.linalg.norm(Gs[1] - Gs[0]) / np.linalg.norm(Gs[0])
    assert rel <= 1e-4


def _requests():
    out = []
    for k, (dims, Re) in enumerate((((200, 80, 1), 40.0), ((320, 96, 1), 80.0),
                                     ((48, 32, 24), 30.0), ((256, 64, 1), 120.0))):
        q = 19 if dims[2] > 1 else 9
        d = serving_porosity(dims, seed=k)
        D = dims[1] / 4.0
        tau = 0.05 * D / Re / (1 / 3) + 0.5
        R = Regions(ffa_x=int(dims[1] / 2 + 5 * D) if dims[1] / 2 + 5 * D < dims[0] - 2 else dims[0] - 3,
                    ffa_y=(0, dims[1]), ffa_z=(0, dims[2]),
                    diss_box=(0, dims[0], 0, dims[1], 0, dims[2]),
                    design_box=(0, dims[0], 0, dims[1], 0, dims[2]))
        out.append(Request(q=q, dims=dims, tau=tau, porosity=d, warm_steps=600, avg_steps=400,
                           objective=H.OBJ_DISSIPATION, max_iter=1000, regions=R, tag=k))
    return out


def test_served_results_identical_alone_and_in_the_mix():
    # the per-request lane (no batching): each request on its own context and stream
    reqs = _requests()
    alone = [solve_one(r) for r in reqs]
    srv = SensitivityServer(slots=4, batch_cells=0)
    futs = [srv.submit(r) for r in reqs]
    mixed = [f.result(timeout=600) for f in futs]
    srv.close()
    for a, m in zip(alone, mixed):
        assert a.J == m.J
        assert a.adjoint_iters == m.adjoint_iters
        assert np.array_equal(a.gradient, m.gradient)


def test_server_rejects_requests_above_the_budget():
    r = _requests()[0]
    srv = SensitivityServer(slots=2, hbm_budget=1 << 20, batch_cells=0)
    fut = srv.submit(r)
    with pytest.raises(H.HlbmError):
        fut.result(timeout=10)
    srv.close()


def test_reused_contexts_give_the_same_results_as_fresh_ones():
    # requests of one grid with different Re: the server reuses idle contexts
    base = _requests()[0]
    reqs = []
    for k, Re in enumerate((30.0, 60.0, 90.0, 45.0, 75.0)):
        D = base.dims[1] / 4.0
        tau = 0.05 * D / Re / (1 / 3) + 0.5
        reqs.append(Request(q=base.q, dims=base.dims, tau=tau, porosity=serving_porosity(base.dims, seed=10 + k),
                            warm_steps=500, avg_steps=300, objective=H.OBJ_DRAG_FFA, max_iter=800,
                            regions=base.regions, tag=k))
    fresh = [solve_one(r) for r in reqs]
    srv = SensitivityServer(slots=2, batch_cells=0)
    got = [f.result(timeout=600) for f in [srv.submit(r) for r in reqs]]
    assert srv.pool.hits >= 1
    srv.close()
    for a, m in zip(fresh, got):
        assert a.J == m.J
        assert np.array_equal(a.gradient, m.gradient)
