"""Failure detection through the C ABI, made on the host side, on a GPU
context that stays usable afterwards (no fault, trap or hang is provoked):

* HLBM_ENOMEM: the caller's allocator hook returns NULL, at creation and at
  the lazy allocation of the adjoint's buffers.
* HLBM_ENONFINITE: a NaN written into the state through hlbm_set_field is
  caught by the primal's device-side check.
* HLBM_EDIVERGED: the adjoint iterated about a mean state whose linearised
  BGK step is unstable (uniform flow at u = 0.35, tau = 0.501: the lattice
  Boltzmann scheme's linear instability at high Mach number and low
  viscosity) grows by more than 1e6 over its smallest residual.

After each error the same context runs the normal path again."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
H = pytest.importorskip("paper_2606_31707_b300.hlbm")
from paper_2606_31707_b300 import Solver  # noqa: E402
from workloads import Regions  # noqa: E402

DIMS = (40, 16, 1)
R = Regions(ffa_x=30, ffa_y=(0, 16), ffa_z=(0, 1), diss_box=(1, 39, 0, 16, 0, 1),
            design_box=(0, 40, 0, 16, 0, 1))


class Hook:
    """Device allocator hook backed by torch's caching allocator that fails
    (returns NULL) once ``budget`` allocations have been made."""

    def __init__(self, budget):
        self.budget = budget
        self.calls = 0
        self.live = set()
        self.alloc = H._ALLOC(self._alloc)
        self.free = H._FREE(self._free)

    def _alloc(self, nbytes, user):
        self.calls += 1
        if self.calls > self.budget:
            return None
        p = torch.cuda.caching_allocator_alloc(int(nbytes), 0)
        self.live.add(p)
        return p

    def _free(self, ptr, user):
        if ptr in self.live:
            self.live.discard(ptr)
            torch.cuda.caching_allocator_delete(ptr)

    def options(self):
        opt = H.hlbm_default_options(DIMS)
        opt.storage = H.FP64
        opt.ffa_x = R.ffa_x
        opt.ffa_y0, opt.ffa_y1 = R.ffa_y
        for k in range(6):
            opt.diss_box[k] = R.diss_box[k]
        opt.dev_alloc = self.alloc
        opt.dev_free = self.free
        return opt


def _porosity():
    y, x = np.mgrid[0:DIMS[1], 0:DIMS[0]]
    d = np.ones((1, DIMS[1], DIMS[0]))
    d[0][(x - 10) ** 2 + (y - 8) ** 2 < 9] = 0.0
    return d.ravel()


def test_enomem_at_create_leaves_no_context():
    hook = Hook(budget=0)
    with pytest.raises(H.HlbmError) as e:
        H.hlbm_create(9, DIMS, 0.7, 0.0, hook.options())
    assert e.value.status == H.ENOMEM
    assert not hook.live


def test_enomem_at_the_lazy_adjoint_allocation_then_recovers():
    # count what creation and the first averaging window allocate, then let
    # the adjoint's first allocation fail
    probe = Hook(budget=10 ** 6)
    ctx = H.hlbm_create(9, DIMS, 0.7, 0.0, probe.options())
    H.hlbm_set_porosity(ctx, _porosity())
    H.hlbm_run_primal(ctx, 200, 10)
    before_adjoint = probe.calls
    H.hlbm_solve_adjoint(ctx, H.OBJ_DRAG_FFA, H.ADJ_EXACT, 1e-8, 20000)
    assert probe.calls > before_adjoint  # the adjoint does allocate lazily
    H.hlbm_destroy(ctx)
    assert not probe.live

    hook = Hook(budget=before_adjoint)
    ctx = H.hlbm_create(9, DIMS, 0.7, 0.0, hook.options())
    H.hlbm_set_porosity(ctx, _porosity())
    H.hlbm_run_primal(ctx, 200, 10)
    with pytest.raises(H.HlbmError) as e:
        H.hlbm_solve_adjoint(ctx, H.OBJ_DRAG_FFA, H.ADJ_EXACT, 1e-8, 20000)
    assert e.value.status == H.ENOMEM
    # the context is still usable: with memory available again the solve runs
    hook.budget = 10 ** 6
    st, it, res = H.hlbm_solve_adjoint(ctx, H.OBJ_DRAG_FFA, H.ADJ_EXACT, 1e-8, 20000)
    assert st == H.OK and res <= 1e-8
    G = np.empty(DIMS[0] * DIMS[1])
    H.hlbm_gradient(ctx, G)
    assert np.isfinite(G).all()
    H.hlbm_destroy(ctx)
    assert not hook.live


def test_nonfinite_state_is_reported_and_the_context_recovers():
    s = Solver(9, DIMS, 0.7, 0.0, storage=H.FP32, u_in=0.05, regions=R)
    s.set_porosity(_porosity().reshape(s.shape))
    s.run_primal(20, 0)
    good = s.field(H.FIELD_F)
    bad = good.copy()
    bad[3, 0, 7, 21] = np.nan
    s.set_field(H.FIELD_F, bad)
    with pytest.raises(H.HlbmError) as e:
        s.run_primal(2, 0)
    assert e.value.status == H.ENONFINITE
    s.set_field(H.FIELD_F, good)
    s.run_primal(20, 5)
    assert np.isfinite(s.field(H.FIELD_F)).all()
    assert np.isfinite(s.objective(H.OBJ_DRAG_FFA))
    s.close()


def _uniform_fbar(s, ux, uy):
    """f^eq(1, u) everywhere, in the library's direction order."""
    xi, w = s.xi.astype(np.float64), s.w
    cu = xi[:, 0] * ux + xi[:, 1] * uy
    uu = ux * ux + uy * uy
    feq = w * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * uu)
    return np.broadcast_to(feq[:, None, None, None], (s.q,) + s.shape).copy()


def test_diverging_adjoint_is_reported_and_the_context_recovers():
    s = Solver(9, DIMS, 0.501, 0.0, storage=H.FP64, u_in=0.05, regions=R, check_every=20)
    s.set_porosity(np.ones(s.shape))
    s.run_primal(4, 2)
    s.set_field(H.FIELD_FBAR, _uniform_fbar(s, 0.35, 0.175))
    with pytest.raises(H.HlbmError) as e:
        s.solve_adjoint(H.OBJ_DRAG_FFA, H.ADJ_EXACT, 1e-10, 5000)
    assert e.value.status == H.EDIVERGED
    # a stable mean state on the same context: the adjoint runs again
    s.set_field(H.FIELD_FBAR, _uniform_fbar(s, 0.05, 0.0))
    st, it, res = s.solve_adjoint(H.OBJ_DRAG_FFA, H.ADJ_EXACT, 1e-10, 200000)
    assert st == H.OK
    assert np.isfinite(s.gradient()).all()
    s.close()
