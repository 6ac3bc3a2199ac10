"""Plain FP64 CPU oracle for the Richardson(m) family (test infrastructure).

This package is test infrastructure, not product code. Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline / reference legs of
``bench.py`` may import it. It shares no code with the CUDA library: the
operators are assembled element by element (Q1) or row by row (Helmholtz)
as sparse matrices, and every iteration is written in the paper's own form
(Table 1 velocity form, eqs. 2-5, 8-9, 14-17, 19-20), with library routines
(sparse mat-vec, dense solve, FFT, autograd) used only as single steps.

Modules
  operators   anisotropic Q1 FEM matrix (Sec. 2.4, eq. 18) and the Helmholtz
              5-point matrix with a first-order absorbing boundary (eq. 22)
  iterations  Richardson(m), MOM/NAG/NAGex-Richardson(m) (Table 1),
              preconditioned form (eq. 17) with the Jacobi and SSOR
              preconditioners, Chebyshev weights (eqs. 8-9),
              residual (eq. 15) and solve-to-tolerance, FP64 refinement split
  training    loss (log form of eq. 15), its gradient, meta MLP, Adam (Alg. 1)
  fourier     two-level step with a Fourier-domain correction (eqs. 19-20)

Parity status of every function is stated in its docstring ("pinned by" or
"parity unpinned").
"""
