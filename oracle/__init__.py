"""Oracle: a plain, slow, FP64 CPU restatement of the IRK monolithic-multigrid method.

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
baseline leg of the benchmark may import this package.  It shares no code with
the CUDA library (no kernels, headers, tables or helpers) and imports nothing
from it; both sides read the same seeded inputs from the `synth` module.

Every function cites the passage of Abu-Labdeh, MacLachlan & Farrell,
"Monolithic multigrid for implicit Runge-Kutta discretizations of
incompressible fluid flow" (arXiv:2202.07381) that it follows.

Parity status per part (what pins it is in tests/test_oracle_*.py):
  tableau      pinned (closed form, order conditions, stability function)
  mesh/numbers pinned (counts, geometry, nesting)
  fem          pinned (independent quadrature, exact identities, MMS orders)
  stage        pinned (scalar Dahlquist reduction, Kronecker identity, time order)
  transfer     pinned (polynomial reproduction, Galerkin identity P^T J_f P = J_c)
  vanka        pinned (explicit-matrix brute force, hand-counted patch sizes)
  colouring    pinned (validity checker, greedy-order definition)
  mg / fgmres  pinned (agreement with a sparse direct solve, mesh-flat iterations)
  local        pinned (rows and patch systems equal those of the assembled J,
               Vanka entries equal the global correction; used for sampled
               checks of the GPU path at sizes where J is not assembled)
"""
