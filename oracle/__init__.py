"""Plain FP64 CPU oracle of matrix-free Neo-Hookean hyperelasticity on Q_p hexahedra.

TEST INFRASTRUCTURE ONLY.  This package is the slow, obviously correct
definition that the CUDA library is checked against.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
it; the library itself never does, and it shares no code with the library.

Everything here is written from the paper (arXiv 2204.01722, "Performance-
Portable Solid Mechanics via Matrix-Free p-Multigrid"):

* ``basis``   -- 1-D Gauss-Legendre / Gauss-Lobatto rules and Lagrange
                 tabulations B_I, B_xi (Sec. II-B, Eq. tensorDense).
* ``fem``     -- structured hexahedral spaces, element restriction, trilinear
                 geometry, kinematics, residual (Eq. variational-form,
                 Eq. Kirchhoff-stress, Eq. residual-discrete), Jacobian action in
                 the paper's current-configuration form (Eqs. Jacobian, dtau,
                 depsilon) and in the initial-configuration form dP = dF S + F dS
                 (Sec. V-E, Table different-storage), operator diagonal and the
                 p-prolongation (Eq. mg_prolong).
* ``solvers`` -- CG with Lanczos estimates, Chebyshev-Jacobi smoothing,
                 the p-multigrid V-cycle (Algorithm multigrid_algorithm) and the
                 load-stepped Newton-Krylov solve (Sec. III-A).
* ``learned`` -- FP64 forward/backward of the small 3-D convolution network
                 used as a learned coarse correction (not in the paper).

Dense Kronecker-product element matrices are used instead of sum
factorisation: the definitions are applied literally, element by element
(batched over elements with numpy), so a reader can check them by eye.
"""
