"""Plain, slow FP64 CPU oracle for the extrapolated geometric-multigrid IGA solver.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.  The
product path (the CUDA library and its Python binding) never imports, links or
calls anything here, and this package imports nothing from the product.

It follows the paper (Mouhssine, Ratnani, Sadok, "Vector extrapolation methods
applied to geometric multigrid solvers for isogeometric analysis", 2024) step
by step, in the paper's order and notation:

* ``bspline``       -- open knot vectors and the Cox-de Boor recursion (Sec. 2.3,
                       Eq. moneq, Prop. 3); Gauss-Legendre rules.
* ``galerkin``      -- Galerkin mass/stiffness factors, the tensor-product
                       operator A^h of Eq. (2), load vectors, L2 projection
                       prolongation P (Sec. 2) and the continuous L2 error.
* ``multigrid``     -- smoothers (multicolour Gauss-Seidel, weighted Jacobi)
                       and the mu-cycle of Algorithm 2 (V-cycle for mu = 1).
* ``extrapolation`` -- RRE (Algorithm 3) and MPE (Algorithm 4) through a QR
                       factorisation, the Schur (Eq. extrapolapprox) and
                       pseudo-inverse (Eq. rreapproxim) forms, and the
                       restarted method of Algorithm 5.
* ``krylov``        -- textbook Arnoldi GMRES / FOM, used only as an
                       independent pin of RRE / MPE.

Every function is pinned by ``tests/test_oracle_*.py`` against values the
paper prints, closed forms, invariants or brute force.  Parity unpinned: the
GS-smoothed cycle counts (the paper reports only Jacobi-smoothed counts, which
the tests check loosely), see the individual module headers.
"""
