"""hlbm_objective_noalloc against the context entry points.

The no-allocation entry point serves callers that must not allocate device
memory (fixed arenas or pools, latency-critical loops, plug-in hosts).  Its
result must equal what a context computes for the same state: J from
hlbm_objective and dJ/df, dJ/dd from hlbm_get_field after a one-sample
window.  Two calls in a row check that the shared scratch array left over
from one call does not leak into the next.  This file is collected last so
that a run stopping at the first failure has run every other test.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
H = pytest.importorskip("paper_2606_31707_b300.hlbm")
from paper_2606_31707_b300 import Solver  # noqa: E402

TOL = 1e-12  # FP64 storage and arithmetic on both sides; only the summation order differs


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("lattice,dims,Cs", [(9, (300, 40, 1), 0.0), (19, (140, 12, 6), 0.12)])
def test_noalloc_objective_matches_context(lattice, dims, Cs):
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    dev = torch.device("cuda", 0)
    nx, ny, nz = dims
    N = nx * ny * nz
    tau, u_in = 0.7, 0.05
    rng = np.random.default_rng(7)
    d = np.clip(rng.uniform(-0.2, 1.2, size=N), 0.0, 1.0)
    # a non-trivial canonical state: equilibrium of a random flow, then a few steps
    s = Solver(lattice, dims, tau, Cs, storage=H.FP64, u_in=u_in)
    D = 2 if lattice == 9 else 3
    u = np.zeros((D, N))
    u[0] = u_in * (1 + 0.3 * rng.standard_normal(N))
    u[1] = 0.02 * rng.standard_normal(N)
    s.set_porosity(d)
    H.hlbm_init_equilibrium(s.ctx, None, u)
    s.run_primal(5, 0)
    f = s.field(H.FIELD_F).reshape(lattice, N)
    s.close()

    f_dev = torch.from_numpy(np.ascontiguousarray(f)).to(dev)
    d_dev = torch.from_numpy(d).to(dev)
    regions = {H.OBJ_DRAG_FFA: (nx // 2, nx // 2 + 1, 1, ny - 1, 0, nz),
               H.OBJ_DISSIPATION: (2, nx - 5, 0, ny, 0, nz)}
    for obj, reg in regions.items():
        # reference: the context entry points on the same state, one-sample window
        from workloads import Regions
        R = Regions(ffa_x=regions[1][0], ffa_y=regions[1][2:4], ffa_z=regions[1][4:6],
                    diss_box=regions[2], design_box=(0, nx, 0, ny, 0, nz))
        c = Solver(lattice, dims, tau, Cs, storage=H.FP64, u_in=u_in, regions=R)
        c.set_porosity(d)
        c.set_field(H.FIELD_F, f.reshape((lattice,) + c.shape))
        c.run_primal(1, 1)
        J_ref = c.objective(obj)
        g_ref = c.field(H.FIELD_GBAR_FFA if obj == H.OBJ_DRAG_FFA else H.FIELD_GBAR_DISS).reshape(lattice, N)
        dd_ref = c.field(H.FIELD_DJDD_FFA if obj == H.OBJ_DRAG_FFA else H.FIELD_DJDD_DISS).reshape(N)
        c.close()
        for call in range(2):
            J = torch.full((1,), np.nan, dtype=torch.float64, device=dev)
            g = torch.zeros((lattice, N), dtype=torch.float64, device=dev)
            dd = torch.zeros(N, dtype=torch.float64, device=dev)
            st = H.hlbm_objective_noalloc(lattice, dims, tau, Cs, u_in, obj, reg, f_dev, d_dev, J,
                                          g, dd, stream=0)
            assert st == H.OK, (call, st)
            torch.cuda.synchronize()
            assert abs(J.item() - J_ref) <= TOL * max(abs(J_ref), 1e-300), (call, J.item(), J_ref)
            assert _rel(g.cpu().numpy(), g_ref) <= TOL
            if obj == H.OBJ_DISSIPATION:
                assert _rel(dd.cpu().numpy(), dd_ref) <= TOL
            else:
                assert np.abs(dd.cpu().numpy()).max() == 0.0


def test_noalloc_rejects_regions_beyond_the_scratch_limit():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import ctypes as C
    dev = torch.device("cuda", 0)
    dims = (256, 300, 300)  # 2 x 300 x 300 = 180000 blocks > 65536
    f = torch.zeros(1, dtype=torch.float64, device=dev)
    J = torch.zeros(1, dtype=torch.float64, device=dev)
    # the Python wrapper refuses buffers smaller than the grid, so the C entry
    # point is called directly: it checks the scratch limit before it launches
    # anything, so the 1-element buffers are never read
    p = C.c_void_p(f.data_ptr())
    st = H.lib().hlbm_objective_noalloc(19, (C.c_int * 3)(*dims), 0.6, 0.0, 0.05, None,
                                        H.OBJ_DISSIPATION, (C.c_int * 6)(0, 256, 0, 300, 0, 300),
                                        p, p, C.c_void_p(J.data_ptr()), None, None, None)
    assert st == H.ESCRATCH
