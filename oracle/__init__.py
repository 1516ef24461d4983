"""FP64 CPU oracle of the HLBM mean-flow adjoint hot path.

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow reference that
the CUDA path is checked against.  Only the tests, the smoke check of the
build entry point and the CPU-baseline leg of the benchmark may import it;
the product package never does, and it imports nothing from the product.

It follows the paper (Ito, Grafen, Bukreev, Kummerlaender, Krause,
"Mean-Flow Adjoint Sensitivity Analysis of Unsteady Flow Around Porous
Cylinders Using a Homogenized Lattice Boltzmann Method"):

* ``lattice``    -- D2Q9 / D3Q19 velocity sets and weights (Sec. 2.1).
* ``hlbm``       -- moments, porous equilibrium, Smagorinsky relaxation time,
                    BGK collision, streaming, boundary nodes (Eq. 2-6, Eq. 8-9
                    and the tau_eff equation of Sec. 2.2).
* ``objectives`` -- far-field drag J_FFA and dissipation J_DISS with their
                    partial derivatives (Sec. 4.2, 4.3).
* ``meanflow``   -- primal run with tracking averages (Eq. averageObjective,
                    Sec. 3.3).
* ``adjoint``    -- local Jacobians of the collision, the assembled step
                    Jacobian, the (mean-flow) adjoint iteration and the
                    gradient (Eq. adjoint_steady / adjoint_unsteady and
                    gradients_steady / gradients_unsteady, Algorithm 1).

Everything is float64 numpy (and scipy.sparse for the assembled Jacobian).
Readings of points the paper leaves open are stated where they are used.

Parity pins: every function here is pinned by a ``-m "not gpu"`` test
against something other than itself (closed forms, invariants, central
finite differences, sparse direct solves, symmetry).  The FTA variant for
C_S > 0 and the mean-flow gradient of unsteady cases have no ground truth
beyond those pins of their parts ("parity unpinned" as end-to-end values:
the mean-flow linearisation is itself an approximation, App. A).
"""
