"""Plain FP64 CPU oracle for the SIPG hybrid-multigrid hot path (arXiv:1910.01900).

TEST INFRASTRUCTURE ONLY.  This package is the slow, obviously-correct reference
that the CUDA library is checked against.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s ``cpu_baseline`` / ``--impl
reference`` leg may import it.  The product path (``paper_1910_01900_gb300``)
never imports, links or executes anything here, and nothing here imports the
product package: the two share no code.

Layout (each function cites the passage of the paper it follows):

* ``basis``     -- 1D Gauss-Lobatto nodes, Gauss-Legendre rule, Lagrange basis
                   (Section 2, "Lagrange polynomials ... Legendre-Gauss-Lobatto
                   nodes", "Gaussian quadrature with p+1 points").
* ``mesh``      -- structured hex box, affine or degree-3 curved mapping x(xi)
                   from the reference cell [0,1]^3 (Section 2; Section 5.3
                   "element mappings of polynomial degree 3").
* ``dg``        -- SIPG bilinear form (Eqs. WeakFormDG, InteriorPenaltyFlux1/2,
                   BoundaryConditions, penalty tau_e), assembled CSR and a naive
                   matrix-free apply with dense reference matrices.
* ``fe``        -- continuous FE Laplacian (Eq. WeakFormFE) with strong
                   Dirichlet constraints kept as identity rows.
* ``transfer``  -- c-, p- and h-transfers as explicit sparse matrices built from
                   1D mass matrices (Section 3.2, L2-orthogonal projection).
* ``multigrid`` -- Chebyshev-Jacobi (Algorithm 3), eigenvalue estimate by 20 CG
                   iterations, V-cycle (Algorithm 2), CG (Algorithm 1) and
                   flexible CG, dense Cholesky coarse solve.
* ``unstructured`` -- SIPG operator on general hexahedral meshes (connectivity
                   from shared vertices, face points paired by physical
                   position, per-face boundary conditions).
* ``amg``       -- smoothed-aggregation AMG and the AMG-preconditioned CG
                   coarse-grid solver (Section 3.3, "Coarse-grid solver").
* ``mlp``       -- CPU reference of the learned per-element smoother network.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
except where its docstring says "parity unpinned".
"""
