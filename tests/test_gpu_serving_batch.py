"""The batched serving lane: several requests stepped together through the
library's batched entry points (one launch per primal step or adjoint sweep
for the whole cohort, a device work list of (context, block) tiles).

* Each result is bitwise the same alone (a cohort of one) and in a mixed
  cohort of different grids, parameters and porosity fields.
* The batched kernels compute what the single-context ones compute: results
  agree with the plain one-solve-per-launch path to FP32 rounding.
* A served gradient against the FP64 oracle's gradient of the same request
  (same steps, window and adjoint iteration count), within 1e-3.
* Contexts a batch cannot hold are rejected with HLBM_EINVAL."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
H = pytest.importorskip("paper_2606_31707_b300.hlbm")
from oracle import adjoint as oadj  # noqa: E402
from oracle import hlbm as ohlbm  # noqa: E402
from oracle import meanflow as omf  # noqa: E402
from oracle import objectives as oobj  # noqa: E402
from paper_2606_31707_b300 import Solver  # noqa: E402
from paper_2606_31707_b300.serve import BATCH_BLOCK_X, Request, SensitivityServer, solve_one  # noqa: E402
from tests.hlbm_cases import direction_perm, rel_l2  # noqa: E402
from workloads import Regions, serving_porosity  # noqa: E402


def _request(dims, Re, seed, objective, warm=600, avg=400, max_iter=1200, tag=None):
    q = 19 if dims[2] > 1 else 9
    D = dims[1] / 4.0
    tau = 0.05 * D / Re * 3.0 + 0.5
    fx = int(min(dims[0] - 3, dims[1] / 2 + 5 * D))
    R = Regions(ffa_x=fx, ffa_y=(0, dims[1]), ffa_z=(0, dims[2]),
                diss_box=(0, dims[0], 0, dims[1], 0, dims[2]),
                design_box=(0, dims[0], 0, dims[1], 0, dims[2]))
    return Request(q=q, dims=dims, tau=tau, porosity=serving_porosity(dims, seed), warm_steps=warm,
                   avg_steps=avg, objective=objective, max_iter=max_iter, regions=R, tag=tag)


def _mix():
    return [_request((200, 80, 1), 40.0, 1, H.OBJ_DRAG_FFA, tag=0),
            _request((320, 96, 1), 80.0, 2, H.OBJ_DISSIPATION, tag=1),
            _request((256, 64, 1), 120.0, 3, H.OBJ_DRAG_FFA, tag=2),
            _request((120, 48, 1), 25.0, 4, H.OBJ_DISSIPATION, tag=3),
            _request((48, 32, 24), 30.0, 5, H.OBJ_DRAG_FFA, tag=4),
            _request((40, 24, 16), 50.0, 6, H.OBJ_DISSIPATION, tag=5)]


def _serve(reqs):
    srv = SensitivityServer(slots=4, batch_cells=400_000)
    futs = [srv.submit(r) for r in reqs]
    out = [f.result(timeout=600) for f in futs]
    cohorts = list(srv.cohorts)
    srv.close()
    return out, cohorts


def test_batched_results_identical_alone_and_in_the_mix():
    reqs = _mix()
    alone = [_serve([r])[0][0] for r in reqs]
    mixed, cohorts = _serve(reqs)
    assert max(cohorts) >= 2   # requests were actually stepped together
    for a, m in zip(alone, mixed):
        assert a.J == m.J
        assert a.adjoint_iters == m.adjoint_iters and a.status == m.status
        assert np.array_equal(a.gradient, m.gradient)


def test_batched_lane_agrees_with_the_plain_path():
    reqs = _mix()
    served, _ = _serve(reqs)
    for r, s_ in zip(reqs, served):
        import dataclasses
        p = solve_one(dataclasses.replace(r, block_x=BATCH_BLOCK_X))
        assert p.adjoint_iters == s_.adjoint_iters
        assert abs(p.J - s_.J) <= 1e-6 * abs(p.J)
        assert rel_l2(s_.gradient, p.gradient) <= 1e-5


def test_served_gradient_matches_the_oracle():
    # a small steady request, the same steps, window and sweep count on both sides
    r = _request((120, 48, 1), 25.0, 4, H.OBJ_DISSIPATION, warm=300, avg=100, max_iter=400)
    r.tol = 0.0
    (res,), _ = _serve([r])
    P = ohlbm.Params(9, r.dims, tau0=r.tau, u_in=r.u_in)
    out = omf.run_primal(ohlbm.initial_state(P), r.porosity, P, r.warm_steps + r.avg_steps,
                         r.avg_steps, r.regions, oobj.DISS)
    lin = oadj.Linearisation(out["fbar"], r.porosity, P, oadj.EXACT)
    lam, _, _ = oadj.solve_adjoint(lin, out[("gbar", oobj.DISS)], tol=0.0, max_iter=res.adjoint_iters)
    G = oadj.gradient(lin, lam, out[("dJdd_bar", oobj.DISS)])
    assert res.adjoint_iters == 400
    assert rel_l2(res.gradient, G) <= 1e-3
    assert abs(res.J - out[("Jbar", oobj.DISS)]) <= 1e-5 * abs(out[("Jbar", oobj.DISS)])


def test_batch_rejects_contexts_it_cannot_hold():
    stream = torch.cuda.Stream()
    sp = int(stream.cuda_stream)
    b = H.hlbm_batch_create(9, sp)
    dims = (64, 16, 1)
    ok = Solver(9, dims, 0.7, 0.0, storage=H.FP32, stream=sp, block_x=128)
    for kw in (dict(storage=H.FP64, stream=sp, block_x=128),      # storage
               dict(storage=H.FP32, stream=sp, block_x=32),       # block width
               dict(storage=H.FP32, block_x=128)):                # another stream
        bad = Solver(9, dims, 0.7, 0.0, **kw)
        with pytest.raises(H.HlbmError) as e:
            H.hlbm_batch_run_primal(b, [ok.ctx, bad.ctx], 2, 0)
        assert e.value.status == H.EINVAL
        bad.close()
    les = Solver(9, dims, 0.7, 0.1, storage=H.FP32, stream=sp, block_x=128)
    with pytest.raises(H.HlbmError):
        H.hlbm_batch_run_primal(b, [ok.ctx, les.ctx], 2, 0)
    # the accepted context still steps
    H.hlbm_batch_run_primal(b, [ok.ctx], 4, 2)
    assert np.isfinite(ok.objective(H.OBJ_DRAG_FFA))
    les.close()
    ok.close()
    H.hlbm_batch_destroy(b)
