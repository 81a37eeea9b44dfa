"""FP64 CPU oracle for the curl-div IgA solve (test infrastructure only).

This package is the slow, plain reference that the CUDA path is checked
against.  Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import it; the product path never does.  It shares no
code with the CUDA library: it evaluates B-splines with the Cox-de Boor
recursion, integrates with Gauss-Legendre quadrature, assembles the d-D
Galerkin matrix directly from the bilinear form, and solves with SciPy.

Modules
-------
bspline   Section 3.1: knots, Cox-de Boor recursion, derivative formula,
          cardinal B-splines in exact rational arithmetic.
iga1d     Section 3.2: mass / advection / stiffness matrices (eq:matr_M,
          eq:matr_A, eq:matr_S) and the Toeplitz factor of the preconditioner
          T (eq:kron_precond).
assemble  Section 4: the d-D curl-div matrix assembled from the bilinear form
          (eq:curl-div) by quadrature, the printed Kronecker forms
          (eq:matr_Amu, eq:matr_Amu3D), load vectors for manufactured
          solutions (Section 6.2).
symbols   Theorem 3.1, Lemma 3.2, Theorems 5.1 / 5.5, eq:lapl2D / eq:lapl3D.
solvers   Section 6: CG, Gauss-Seidel, the Galerkin V-cycle with the block
          prolongator (eq:2by2prol), PCG / PGMRES post-smoothing with T,
          and the strategies MIM, P_MIM, P_WL.
          (solvers also holds D^{-1} and the generalized eigenpairs by their
          plain definitions: sparse LU and dense LAPACK.)

Parity status: every function here is pinned by a ``-m "not gpu"`` test
against values the paper fixes or mathematics fixes (see tests/test_oracle_*.py);
none is "parity unpinned".
"""
