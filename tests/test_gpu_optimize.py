"""The projected-gradient porosity optimiser built on the adjoint gradient
(the paper's future-work loop): J decreases monotonically, the porosity stays
in [0, 1] and the design-box mean is kept."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

H = pytest.importorskip("paper_2606_31707_b300.hlbm")
from paper_2606_31707_b300 import Solver  # noqa: E402
from paper_2606_31707_b300.optimize import optimise  # noqa: E402
from workloads import Regions, grf_porosity  # noqa: E402


def test_optimiser_decreases_dissipation():
    dims = (160, 64, 1)
    box = (40, 70, 17, 47)
    d0 = grf_porosity(dims, box, corr=3.0, seed=5)
    R = Regions(ffa_x=120, ffa_y=(0, 64), ffa_z=(0, 1), diss_box=(0, 160, 0, 64, 0, 1),
                design_box=(box[0], box[1], box[2], box[3], 0, 1))
    s = Solver(9, dims, 0.8, 0.0, storage=H.FP64, u_in=0.05, regions=R)
    res = optimise(s, d0, H.OBJ_DISSIPATION, primal_steps=6000, iterations=4, step=0.3, tol=1e-9)
    s.close()
    h = res.history
    assert len(h) >= 3
    assert all(b < a for a, b in zip(h, h[1:]))
    d = res.porosity
    assert d.min() >= 0.0 and d.max() <= 1.0
    sl = (slice(0, 1), slice(box[2], box[3]), slice(box[0], box[1]))
    assert np.array_equal(d[:, :, :box[0]], d0[:, :, :box[0]])
    assert abs(d[sl].mean() - d0[sl].mean()) < 0.05
