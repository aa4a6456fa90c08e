"""CPU FP64 oracle for the node-parallel diagonal IMEX SDC sweep (test infrastructure).

This package is test infrastructure.  Only the tests, the smoke check of the
package entry point and the CPU-baseline leg of the benchmark may import it;
the product (the CUDA library and its Python binding) never calls it.

It restates the method of Freese, Götschel, Lunet, Ruprecht & Schreiber,
"Parallel performance of shared memory parallel spectral deferred
corrections" (arXiv 2403.20135), in plain, slow, obviously checkable numpy
FP64 code:

* ``sht``  -- Gauss-Legendre grid, normalised associated Legendre functions,
  naive DFT along longitude, direct Legendre sums (Sec. 3.2: the
  spherical-harmonic transform that the tendencies need).
* ``swe``  -- the shallow-water operators in vorticity-divergence form:
  the implicit gravity term L_g and the explicit T_E = L_c + N_a + N_r of
  Eq. (4), and the per-mode solve u - alpha L_g(u) = beta of Eq. (8) by
  dense Gaussian elimination.
* ``sdc``  -- Radau-right collocation nodes, the collocation matrix Q, the
  MIN-SR-FLEX diagonal coefficients (Sec. 4.2) and the dSDC step of
  Algorithm 2 built on the node update of Eq. (7).

Library primitives (numpy matmul, LAPACK solves, polynomial roots) serve as
single steps; there is no blocking, fusion or reordering beyond the written
definitions.  It shares no code with the CUDA path; only ``swe_inputs``
(seeded inputs, no method arithmetic) serves both.
"""
