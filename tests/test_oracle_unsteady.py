"""Pins of the oracle's checkpointed short-horizon unsteady adjoint (the
validation reference for the exact transient sensitivities of App. C):
central differences of J_T, exactness of the checkpointing, and the duality
identity with the tangent-linear recursion."""
import numpy as np
import pytest

from oracle import adjoint as adj
from oracle import hlbm
from oracle import objectives as obj
from oracle.hlbm import Params
from workloads import Regions, cylinder_porosity


def _case(q=9, Cs=0.0, collision="bgk"):
    dims = (24, 12, 1) if q == 9 else (14, 8, 4)
    P = Params(q, dims, tau0=0.7, Cs=Cs, u_in=0.05, collision=collision)
    d = cylinder_porosity(dims, 7.0, dims[1] / 2.0, 2.0, 1.2, jitter=0.01, seed=3)
    nx, ny, nz = dims
    R = Regions(ffa_x=nx - 5, ffa_y=(0, ny), ffa_z=(0, nz),
                diss_box=(2, nx - 3, 0, ny, 0, nz), design_box=(0, nx, 0, ny, 0, nz))
    return P, d, R


def _JT(f0, d, P, T, objective, R):
    f = f0.copy()
    s = 0.0
    for n in range(T):
        s += obj.value(f, d, P, objective, R) / T
        if n < T - 1:
            f = hlbm.step(f, d, P)
    return s


@pytest.mark.parametrize("q,Cs,collision,T", [(9, 0.0, "bgk", 60), (9, 0.2, "bgk", 40),
                                              (9, 0.1, "rr", 40), (19, 0.0, "bgk", 12)])
@pytest.mark.parametrize("objective", [obj.FFA, obj.DISS])
def test_unsteady_adjoint_vs_central_differences(q, Cs, collision, T, objective):
    P, d, R = _case(q, Cs, collision)
    f0 = hlbm.initial_state(P)
    G, JT, _ = adj.unsteady_adjoint_gradient(f0, d, P, T, objective, R)
    assert abs(JT - _JT(f0, d, P, T, objective, R)) <= 1e-15 * max(1.0, abs(JT))
    rng = np.random.default_rng(5)
    h = 1e-6
    for _ in range(2):
        v = rng.standard_normal(d.shape)
        fd = (_JT(f0, d + h * v, P, T, objective, R) - _JT(f0, d - h * v, P, T, objective, R)) / (2 * h)
        an = float((G * v).sum())
        assert abs(fd - an) <= 1e-7 * max(abs(an), 1e-3 * np.abs(G).sum())


def test_checkpointing_recomputes_the_same_states():
    P, d, R = _case()
    f0 = hlbm.initial_state(P)
    T = 50
    Ga, Ja, fa = adj.unsteady_adjoint_gradient(f0, d, P, T, obj.DISS, R, checkpoint_every=1)
    Gb, Jb, fb = adj.unsteady_adjoint_gradient(f0, d, P, T, obj.DISS, R)
    assert np.array_equal(Ga, Gb) and Ja == Jb
    assert fa == T - 1               # every state stored: no recomputation
    assert fb <= 2 * (T - 1)         # checkpoints every ceil(sqrt(T)): one extra forward pass at most


def test_unsteady_adjoint_duality_with_the_tangent_recursion():
    # <G, delta> = (1/T) sum_n (g_n . v_n + dJ/dd_n . delta),  v_{n+1} = A_n v_n + D_n delta
    P, d, R = _case(9, 0.2)
    f0 = hlbm.initial_state(P)
    T = 30
    G, _, _ = adj.unsteady_adjoint_gradient(f0, d, P, T, obj.DISS, R)
    delta = np.random.default_rng(9).standard_normal(d.shape)
    f = f0.copy()
    v = np.zeros_like(f0)
    acc = 0.0
    for n in range(T):
        g, gd = obj.partials(f, d, P, obj.DISS, R)
        acc += (float((g * v).sum()) + float((gd * delta).sum())) / T
        lin = adj.Linearisation(f, d, P, adj.EXACT, outlet="streamed")
        v = lin.jvp(v) + (lin.D @ delta.ravel()).reshape(f.shape)
        f = hlbm.step(f, d, P)
    assert abs(acc - float((G * delta).sum())) <= 1e-12 * max(1.0, abs(acc))
