"""FP64 CPU oracle for the variable-coefficient staggered Stokes solver.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check of
``__graft_entry__`` and the ``cpu_baseline`` / ``--impl reference`` legs of
``bench.py`` may import this package.  The CUDA path never calls it and shares
no code with it.

Everything here is written from Cai, Nonaka, Bell, Griffith & Donev,
"Efficient Variable-Coefficient Finite-Volume Stokes Solvers" (arXiv:1308.4605):

  grid.py       index maps of the MAC grid (Sec. 3.1)
  assemble.py   D, G, L_mu, rho, M, L_rho as scipy.sparse matrices (Sec. 2, 3.1)
  multigrid.py  coarse coefficients, restriction, prolongation, multicolour
                Gauss-Seidel and the V-cycles (App. C)
  precond.py    the block preconditioners P1..P5 (Sec. 2.1-2.4)
  krylov.py     left-preconditioned GMRES(m) and flexible GMRES (Sec. 3.2, 4)
  direct.py     bordered direct solves of M x = b (the exact discrete solution)
  fourier.py    Fourier-space closed forms for constant coefficients (App. A)
  gradient.py   adjoint gradient of a quadratic velocity loss w.r.t. log mu, rho

Parity status of each function is stated in its module header.
"""
