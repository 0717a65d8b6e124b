"""Reference oracle for the two-level Lippmann-Schwinger solver (test infrastructure).

A plain, slow, FP64 CPU implementation of what the GPU path computes, written
from the paper (Zepeda-Nunez & Zhao, "Fast alternating bi-directional
preconditioner for the 2D high-frequency Lippmann-Schwinger equation").
It is test infrastructure: only the tests, the smoke entry point and the
benchmark's CPU-baseline / reference legs may import it.  The CUDA library
never calls into it and shares no code with it; the only module both use is
the seeded input generator `paper_1602_07652_gb300.inputs`, which holds none
of the method's arithmetic.

Modules
  greens    -- kernel G (eq. Greens_function), corrected-trapezoid weights (Sec. 2),
               Toeplitz/FFT apply of H = I + w^2 G D and the right-hand side f.
  sparsify  -- sparsifying stencil A (Sec. 2, SVD problem), sparsified matrix C.
  polarized -- layered decomposition, local matrices C^l (Sec. 3.1-3.3),
               Algorithm 1 (Gauss-Seidel preconditioner, Sec. 3.4) and
               Algorithm 2 (bi-directional preconditioner, Sec. 3.5).
  krylov    -- restarted flexible GMRES (Sec. 4; FGMRES per Sec. 6).
  solver    -- Algorithm 3 (Lippmann-Schwinger preconditioner, the inner
               level) and the outer iteration on H u = f (Sec. 4).

Every function's docstring cites the passage it follows.  Readings of passages
the paper leaves silent, ambiguous or garbled are stated where they are used.
"""
