"""Plain, slow CPU FP64 oracle of the dual-primal domain-decomposition spectral-element
Helmholtz method (Galagusz & McFee, arXiv 1808.04713).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this package: only
``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference leg
use it.  It shares no code with the CUDA library (``paper_1808_04713_gb300``); the two
meet only through the seeded inputs of ``workloads.py``.

Modules
  legendre     Section 2.1: orthonormal Legendre recurrence, D, S, integrated basis,
               interpolatory basis B, affine re-expansion L (by its defining integral).
  element      Section 2.2.1: tensor-product element operator, Robin terms and loads.
  mesh         quadtree leaves -> sides, master edges, hanging relations, vertices.
  constraints  Section 2.2.4: global constraint matrix C (padded, eq. final_constraint),
               the split C = [C_p; C_d], unknown types (Algorithm 1) and the basis Z.
  direct       the globally assembled conforming solve (null space of C).
  dd           Section 2.3: partial-nullspace dual-primal solve, block inversion with the
               coarse matrix K, Dirichlet preconditioner, FGMRES, recovery.
  adjoint      the adjoint (conjugate) solve and permittivity gradient.
  poisson      Section 3.1: the Poisson test with zero Dirichlet data and rho jumps, the
               Dirichlet preconditioner with diagonal scaling, PCG and the spectrum of
               P^-1 F (pinned to the printed Table 2).
  dirichlet    Section 3.2: the Helmholtz test with point-source Dirichlet data (lifting of
               the boundary trace, zero-data dual-primal solve, FGMRES), pinned to the exact
               solution and to the printed Table 3.
  pml          Section 4: axis-aligned PMLs by complex coordinate stretching (per-element
               anisotropic coefficients on the same split), pinned to the exact stretched plane
               wave and to the layer's absorption.

Parity status: every function is pinned by tests in ``tests/test_oracle_*.py``; see the
docstrings for the pin of each part.
"""
