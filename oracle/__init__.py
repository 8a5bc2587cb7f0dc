"""FP64 CPU oracle for GenEO-preconditioned CG on anisotropic elasticity.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct
restatement of the method of "High-performance dune modules for solving
large-scale, strongly anisotropic elliptic problems with applications to
aerospace composites" (Butler et al., arXiv:1901.05188), written in numpy/scipy
in double precision.  Only the test suite, the smoke check of the package entry
point and the CPU-baseline leg of the benchmark may import it.  It shares no
code with the CUDA path and never imports it.

Modules (each function cites the passage it follows):
  material  -- orthotropic / isotropic Hooke law and tensor rotation (Sec. 2)
  fem       -- Q1 hexahedra, Gaussian integration, assembly, BCs, load,
               element stresses (Sec. 2)
  decomp    -- box partition, overlap, restriction sets, partition of unity
               (Sec. 3.1, Sec. 3.2 Def. of overlap / PoU, Sec. 3.3.1)
  geneo     -- GenEO eigenproblems, coarse space, coarse matrix (Sec. 3.2-3.3),
               and the zero-energy-mode coarse space (Sec. 5, Table 1)
  krylov    -- one- and two-level additive Schwarz, PCG, flexible CG,
               condition estimate (Sec. 3.1), inexact coarse solve (Sec. 3.3.3)
  solver    -- the whole pipeline for one problem
  darcy     -- the scalar Darcy problem of the SPE10 application (Q1, one
               unknown per node)
  serendipity -- 20-node serendipity hexahedra (the paper's element, Sec. 5):
               shape functions, 3x3x3 Gauss stiffness, mesh, face load, and
               the node sets the decomposition and GenEO stages use on it

Every function here is pinned by tests in tests/test_oracle_*.py against
closed forms, invariants and brute force; none is marked "parity unpinned".
"""
