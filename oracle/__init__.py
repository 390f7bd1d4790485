"""Plain, slow, FP64 CPU oracle for the spline geometric leapfrog scheme.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It
shares no code with the CUDA path (``paper_2302_04979_gb300``) and imports
nothing from it.

Every function cites the passage of Kapidani & Vazquez, "High order geometric
methods with splines: fast solution with explicit time-stepping for Maxwell
equations" (arXiv 2302.04979) it follows.  Where the paper reaches a result
with a plain definition (a Kronecker solve reaches x = C^-1 y, a mass apply
reaches y = M x), the oracle writes that definition out with library
primitives (LAPACK LU, sparse matrices, einsum over tensor-product bases).

Modules
-------
splines   univariate knots, B-spline / Curry-Schoenberg bases, 1D pairing
          matrices G-hat and M-hat, 1D incidence (Sec. 2.3, Sec. 4.1)
forms3d   tensor-product layout of the primal and dual complexes, 3D
          incidence D^1, D~^1, D^2, D~^2 and pairing blocks K_1, K~_1
          (Sec. 2.3-2.4, Eq. tensor_K, Eq. tensor_Ktilde)
hodge     geometry map, material, matrix-free Hodge mass apply M^2, M~^2
          (Sec. 3.4, 2-form pullback of Sec. 2.3)
maxwell   scheme 2 leapfrog step, energy, CFL by power iteration,
          L2 projection and error norms (Sec. 3.4, Sec. 4.2, Sec. 5)
scheme1   scheme 1: 1-form mass matrices M^1_eps, M~^1_mu and the leapfrog
          with mass-matrix Hodge stars, energy, CFL (Sec. 3.3, Sec. 5.2)
lifting   scheme 2 with a prescribed tangential trace of E: the whole spaces
          X^1_h, X^2_h, the local projection of the boundary data, and the
          lifted leapfrog (Sec. 3.5, Sec. 5.1.2)
adjoint   the discrete adjoint of the scheme-2 step (a derivative of the
          discrete map, not a passage of the paper)

Parity status: every function is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_*.py`` against closed forms, identities the paper states,
library routines or brute force on tiny meshes.  No function is left
"parity unpinned".
"""
