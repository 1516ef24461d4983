"""Host-side logic, no GPU: the benchmark's algorithmic byte model (the
roofline's numerator) and the serving form's admission bookkeeping."""
import pytest

import bench
from workloads import make_workload


def test_byte_model_of_the_les_case():
    wl = make_workload("les3d_re3900")
    bm = bench.bytes_model(wl, 4, 4, exact_rec=True)
    # plain step: read and write 19 FP32 populations, read the porosity
    assert bm["plain"] == 2 * 19 * 4 + 4
    # exact LES adjoint: lambda read and written, the record f_bar - w, the
    # porosity, plus the two drag coefficients on the plane (1 of 640 columns)
    assert bm["adj_ffa"] == pytest.approx((2 * 19 + 19 + 1) * 4 + 2 * 4 / 640, rel=1e-12)
    # averaging: the 19 sums of f - w and tau_eff - tau0 staged in FP32 (8 B per
    # sample, a 24 B FP64 fold every 64 samples), plus region terms
    per_sum = 8 + 24 / 64
    assert bm["acc"] > bm["plain"] + 20 * per_sum
    assert bm["acc"] == pytest.approx(397.23, abs=0.01)
    # FP16 deviations halve the population bytes of the plain step
    assert bench.bytes_model(wl, 2, 4, exact_rec=True)["plain"] == 2 * 19 * 2 + 4


def test_slab_has_the_bytes_per_update_of_the_full_grid():
    # the ncu captures run on the 24-deep slab and are scaled by the cell ratio
    full = bench.bytes_model(make_workload("les3d_re3900"), 4, 4, exact_rec=True)
    slab = bench.bytes_model(make_workload("les3d_re3900_slab"), 4, 4, exact_rec=True)
    for k in full:
        assert slab[k] == pytest.approx(full[k], rel=1e-4)


def test_measured_traffic_is_below_the_algorithmic_bytes():
    # no kernel re-reads: every stored DRAM figure is at most the algorithmic bytes
    for (h, wname, storage, coll, kernel), traffic in bench.MEASURED_DRAM.items():
        wl = make_workload(wname)
        bm = bench.bytes_model(wl, 4, 4, exact_rec=True)
        key = {"primal_step_accumulate": "acc", "primal_step_plain": "plain",
               "adjoint_step_ffa": "adj_ffa", "adjoint_step_diss": "adj_diss"}[kernel]
        alg = bm[key] * wl.cells
        assert 0.85 * alg <= traffic <= 1.1 * alg, (wname, kernel, traffic / alg)


H = pytest.importorskip("paper_2606_31707_b300.hlbm")
from paper_2606_31707_b300 import serve  # noqa: E402


class _FakeSolver:
    def __init__(self):
        self.closed = False

    def close(self):
        self.closed = True


def test_context_pool_accounts_and_evicts_oldest_first():
    pool = serve.ContextPool()
    a, b = _FakeSolver(), _FakeSolver()
    pool.give(("k", 1), a, 100)
    pool.give(("k", 2), b, 50)
    assert pool.idle_bytes == 150
    assert pool.take(("k", 2)) is b and pool.idle_bytes == 100 and pool.hits == 1
    assert pool.take(("k", 3)) is None and pool.misses == 1
    pool.give(("k", 2), b, 50)
    assert pool.evict_one() and a.closed and not b.closed and pool.idle_bytes == 50
    pool.clear()
    assert b.closed and pool.idle_bytes == 0 and not pool.evict_one()


def test_footprint_counts_the_krylov_basis():
    dims = (200, 80, 1)
    fp = serve.footprint_bytes(9, dims, H.FP32)
    gm = serve.footprint_bytes(9, dims, H.FP32, adjoint_solver=1, gmres_restart=30)
    assert gm - fp == (30 + 4) * 9 * 200 * 80 * 4
    assert serve.footprint_bytes(19, (64, 32, 16), H.FP32) > serve.footprint_bytes(9, (64, 32, 1), H.FP32)


def test_only_small_fixed_point_fp32_requests_are_batched():
    import numpy as np

    base = dict(q=9, dims=(200, 80, 1), tau=0.6, porosity=np.ones((1, 80, 200)))
    assert serve.batchable(serve.Request(**base), 400_000)
    assert not serve.batchable(serve.Request(**base, adjoint_solver=1), 400_000)
    assert not serve.batchable(serve.Request(**base, Cs=0.1), 400_000)
    assert not serve.batchable(serve.Request(**base, storage=H.FP64), 400_000)
    assert not serve.batchable(serve.Request(**base), 10_000)
