"""Plain FP64 CPU oracle for the hierarchical multigrid finite cell method.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only the tests, the package's smoke check and the
benchmark's CPU-baseline and reference legs use it.  It shares no code with
the CUDA library; the two meet only through the problem descriptions of
``fcm_inputs`` and the documented degree-of-freedom layout.

Contents, each following the paper (Jomo et al., "Hierarchical multigrid
approaches for the finite cell method on uniform and multi-level hp-refined
grids", arXiv 2010.00881):

* ``basis``       integrated Legendre basis (Sec. 2.1), Gauss-Legendre rules
* ``geometry``    level sets (balls, voids, ellipsoids, the popcorn of
                  Sec. 4.3.2, the rotated square of Sec. 4.1.2), cell
                  classification, whole-grid classification
* ``quadrature``  space-tree cut-cell integration, surface rules
* ``assembly``    element matrices and the global system of Eq. (weakform)
* ``multigrid``   level hierarchy (Eq. restrictionoperation,
                  Eq. hierarchicalMatrices), additive Schwarz smoother
                  (Eq. AdditiveSchwarz; elementwise or patchwise blocks,
                  Sec. 3.3.1; Jacobi and Gauss-Seidel for comparison,
                  Sec. 4.1), V-cycle (Algorithm 1), PCG (Sec. 4), multigrid
                  as a stand-alone solver
* ``mlhp``        multi-level hp overlays (Sec. 2.2): overlay mesh, active
                  basis, leaf assembly, hp-multigrid levels (Sec. 3.2,
                  Fig. hpmultigrid) with patchwise blocks over base cells
* ``trunk``       trunk-space elements (the paper's 3D space, Table
                  tab::upperbound) as a mask on the tensor layout, removal of
                  fully fictitious cells, their p- and h-multigrid

Pins (tests/test_oracle_*.py) tie each function to something other than
itself; see the module docstrings.
"""
