"""Oracle: a plain, slow, FP64 CPU restatement of the method of Alexandersen & Lazarov,
"Robust topology optimisation of microstructural details without length scale separation
-- using a spectral coarse basis preconditioner" (arXiv:1411.3923).

This package is TEST INFRASTRUCTURE.  Only the test-suite, the smoke check and the
CPU-baseline leg of the benchmark may import it.  The CUDA library never imports, links or
calls it, and it shares no code, tables or constants with the CUDA library.

Modules
-------
fem       Q4 plane-stress discretisation, assembly, boundary conditions, direct solve
          (Sec. 2.1-2.2)
design    density filter, Heaviside projection, SIMP, compliance sensitivities, robust
          combination and the filter transpose (Sec. 2.2, 4.1-4.4)
msfem     agglomerates, local generalised eigenproblems with diagonal weighting, partition
          of unity, coarse basis R_c and K_c, overlapping patch solves, the additive
          two-level preconditioner and PCG (Sec. 2.4, 3.2)
smoother  the paper's own preconditioner: symmetric Gauss-Seidel before and after the
          spectral coarse solve, applied multiplicatively (Sec. 2.4.2), with the
          lexicographic point sweep and the GPU's colour-by-colour node-block sweep, and
          the paper's outer method, right-preconditioned restarted GMRES
pde_filter  the PDE (Helmholtz) density filter with periodicity and connectivity imposed by
          collapsed DOFs, for designs of several microstructure blocks (Sec. 4.3, 4.5)
optimise  the design loop: MMA (one constraint, dual by bisection) on the robust compliance
          with the expected-volume constraint, and the continuation schedule (Sec. 4.4, 4.5)
pipeline  the whole hot path on one workload (Sec. 5.3 for the shared preconditioner)

Pins: every function here is checked by tests/test_oracle_*.py against closed forms,
invariants, brute force and finite differences.  Parity unpinned: the paper's printed
compliances, timings and iteration counts (they need the paper's optimisation histories).

Conventions (deliberately different from the CUDA library's):
  node (i, j) with i in [0, nelx] along x and j in [0, nely] along y (upwards);
  oracle node number n = i*(nely+1) + j (column-major), DOFs 2n (x) and 2n+1 (y);
  element (ex, ey) has oracle number ex*nely + ey and nodes (ex,ey), (ex+1,ey), (ex+1,ey+1),
  (ex,ey+1) in that order.
Arrays that cross into or out of this package use the neutral layout shared with the
input generators: element fields as [nely][nelx] (row 0 at the bottom), nodal vectors as
[nely+1][nelx+1][2].
"""
