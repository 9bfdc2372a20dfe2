"""FP64 CPU oracle for the statically condensed spectral-element Helmholtz solver.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and
its Python binding) may import, call or link anything in this package.  Only
the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use it.

It is written from the paper's definitions (Huismann, Stiller, Froehlich,
"Factorizing the factorization", arXiv:1601.08179), slowly and plainly:

* ``gll``       -- 1D Gauss-Lobatto-Legendre nodes, weights, lumped mass M and
                   stiffness K (Sec. 3).
* ``element``   -- metric coefficients d_e (Eq. metriccoeffelement) and the
                   dense element operator H_e as a sum of Kronecker products
                   (Eq. helmholtz_operator).
* ``mesh``      -- Cartesian mesh, global node numbering, the packed skeleton
                   layout (faces, edges, vertices) declared in include/sem.h.
* ``dense``     -- assembled operators on tiny meshes: the full system
                   R H_L R^T, the dense Schur complement H_BB - H_BI H_II^-1 H_IB
                   per element (Eqs. condensation_inner/condensation_system),
                   condensed right-hand side, interior recovery (Algorithm 1),
                   brute-force direct solves.
* ``local``     -- the same condensed operator, element by element, with the
                   Kronecker blocks applied as mode products and H_II^-1 by the
                   tensor-product eigendecomposition (Sec. 5); vectorised over
                   elements so that it runs at full benchmark sizes.
* ``transform`` -- the coordinate transform S = diag(1, S_II, 1) of Sec. 6 on
                   the skeleton, with a canonical eigenvector choice.
* ``pcg``       -- Hestenes-Stiefel preconditioned conjugate gradients (Sec. 8).
"""
