"""Plain FP64 CPU oracle for the IEDG per-element local problem.

This package is TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
The product path (the CUDA library and its Python binding) never imports, links or
executes anything here, and nothing here imports the product path.

What it computes, written from the paper (Fernandez, Nguyen, Roca, Peraire,
"Implicit large-eddy simulation of compressible flows using the Interior
Embedded Discontinuous Galerkin method", arXiv:1605.01020):

* ``refelem``  -- reference element: Gauss-Legendre / Gauss-Lobatto-Legendre
  points by Newton iteration, tensor Lagrange basis (Sec. 2.1, the spaces the
  IEDG form is posed in).
* ``geometry`` -- isoparametric map of degree p = k (Sec. 3.1), Jacobians,
  scaled face normals.
* ``physics``  -- compressible Navier-Stokes fluxes (Eq. NS and the flux /
  stress / heat-flux / pressure definitions of Sec. 2.1), Lax-Friedrichs
  numerical flux (Eq. IEDG d), pointwise Jacobians by forward-mode dual numbers.
* ``iedg``     -- residuals R_NS, R_FL (Eq. IEDG a-c, Eq. NLS), Jacobian blocks
  A, B, C, D and right-hand sides F, G (Newton system, Sec. 2.2.1), static
  condensation K = D - C A^-1 B, R = G - C A^-1 F (Eq. LS) in the full form
  (dense A, the definition) and the q-eliminated form, assembly into a block
  compressed-row trace matrix (Sec. 2.2.2), back-substitution.
* ``bilu``     -- block ILU(0) of the trace matrix and its solve (Sec. 2.2.2).
* ``lowprec``  -- the condensed block with the Schur complement's operands
  rounded to TF32 or BF16 (the reading of a low-precision Schur GEMM).

Every function is FP64, plain numpy/scipy, no blocking or fusion beyond what the
definitions state.  Parity status: every function is pinned by a test in
``tests/test_oracle_*.py`` (closed forms, invariants, finite differences, dense
uncondensed solves, manufactured solutions); conventions the paper leaves open
are listed in the module docstrings and pinned only through those invariants.
"""
