"""Plain, slow FP64 CPU oracle for the phase-field fracture hot path.

TEST INFRASTRUCTURE ONLY. Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package. The product path (the CUDA
library and its Python binding) never imports, links or calls it, and it shares no code
with that path: every formula here is written out from the paper's definitions.

What it computes (paper: Jodlbauer, Langer, Wick, "Parallel matrix-free higher-order
finite element solvers for phase-field fracture problems"):

* ``basis``    -- 1D Gauss-Legendre points, Gauss-Lobatto-Legendre nodes, Lagrange bases (Sec. 3.1).
* ``mesh``     -- uniform Q_p meshes of the unit square / cube, DoF numbering, Dirichlet data of the
                  tension and shear tests, the slit (phi = 0 on its nodes, or cut into the mesh with
                  duplicated nodes), DoF counts of Table tab:slit:dofs:p (Sec. 5.1, 5.2).
* ``material`` -- degradation g, strain, Miehe spectral split, the eigen-derivative of Eqs.
                  (lin_lambda), (lin_v) and Alg. 2, and the tangent of the split stress (Sec. 2.1, 3.5).
* ``fe``       -- the residual of Eq. (residual) and the Jacobian of Eq. (G), both assembled cell by
                  cell from full tensor-product tables (no sum factorisation), the energy of Sec. 2.1,
                  lumped mass, parameter gradients of the residual, the force on the loaded face.
* ``solvers``  -- Alg. 1 (active set, one primal-dual active-set step), transfers between nested
                  meshes, Chebyshev-Jacobi smoothing and eigenvalue estimation (Sec. 3.3), the
                  monolithic V-cycle with block-diagonal smoother, flexible GMRES.

Pins: every function is checked by ``tests/test_oracle_*.py`` against values the paper
prints, closed forms, exact symbolic integration, finite differences or library routines.
The V-cycle is pinned on two levels against the same cycle composed from dense matrices, with
the smoother taken from its closed-form error polynomial; on more levels it is that composition
applied recursively, and it is checked to contract.
"""
