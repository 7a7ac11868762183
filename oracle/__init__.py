"""FP64 CPU oracle for the Wilson-clover solver path (TEST INFRASTRUCTURE).

This package is a plain, slow, obviously correct NumPy restatement of what the
GPU library computes. It exists only to check the GPU path: the tests, the
``smoke()`` check and the benchmark's CPU-baseline leg may import it; the
library itself never does, and this package imports nothing from the library.

Sources of each definition (paper: Gruber et al., "Performance optimizations
for porting the openQ*D package to GPUs", LATTICE2021):

* ``dirac``     - O(a)-improved Wilson-Dirac operator (Sec. 1), its even-odd
                  ordering (Sec. 3, Fig. 3) and Schur complement.  The paper
                  gives no formula; the operator is the standard
                  Wilson + Sheikholeslami-Wohlert one in openQCD normalisation.
* ``precision`` - rounding to the storage formats of Table 1.
* ``solvers``   - CGNE with reset steps (Sec. 2, Fig. 4 caption), SAP with
                  static and adaptive cycle/MR counts (Sec. 3, 3.2) and
                  flexible GCR (Sec. 3.1, Table 2).
* ``ptc``       - gauge-equivariant parallel-transport layers used as a
                  learned preconditioner (not in the paper; built from the
                  definition of parallel transport on the lattice).

Parity of the learned preconditioner's *quality* is unpinned (no published
numbers exist); its forward/backward arithmetic is pinned by exact
equivariance and finite differences.
"""
