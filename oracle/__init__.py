"""FP64 CPU oracle for the DDM-GMRES solve of the time-harmonic Maxwell system.

TEST INFRASTRUCTURE ONLY.  Only `tests/`, `__graft_entry__.smoke()` and the
`cpu_baseline` / `--impl reference` legs of `bench.py` may import this
package.  The CUDA library never calls it and shares no code with it.

Contents (paper = Beuchler, Kinnewig, Wick, "Parallel domain decomposition
solvers for the time harmonic Maxwell equations"):

  fem.py      mesh numbering, curl-conforming bases, element matrices by Gauss
              quadrature, global assembly of Eqs. 2-3, Dirichlet lifting, and
              the monolithic direct solve (the plain definition of the result).
  ddm.py      the non-overlapping optimized-Schwarz DDM of Section 3.1
              (Eqs. 4-6, S = identity), the interface system of Eq. 8 solved by
              GMRES or Jacobi, and subdomain solves that are either direct or
              GMRES with the block preconditioner of Eq. 7.
  krylov.py   textbook right-preconditioned restarted GMRES (Arnoldi + Givens).
  adjoint.py  discrete adjoint of the monolithic solve (no counterpart in the
              paper): gradients w.r.t. per-cell mu^{-1} and omega.

Every function is pinned by `tests/test_oracle_*.py` against something other
than itself (closed forms, exact integer identities, an independent 1-D
finite-element solve, the monolithic solve, finite differences).
"""
