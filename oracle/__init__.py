"""CPU oracle for the gauge-conserving spectral PIC step (test infrastructure only).

This package is a plain, slow, FP64 restatement of the method of Christlieb, Sands
and White, "A PIC method with a generalized-momentum formulation, Part III: a family
of gauge-conserving methods" (arXiv 2410.18414).  It exists so that tests, the
bench's CPU-baseline leg and the package smoke check can compare the CUDA library
against something whose every step a reader can check against the paper by eye.

Rules it keeps:
  * It is test infrastructure.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
    CPU-baseline / reference legs of ``bench.py`` may import it.  The CUDA library
    never calls it and shares no code with it.
  * Everything is numpy float64 / complex128.  Loops run over stencil offsets and
    time levels only; particles and modes are numpy vectors.
  * The DFT is the definition written as a dense matrix product (no FFT).
  * Spline weights come from the Cox-de Boor recursion, not from closed-form
    polynomials.

Modules:
  bspline   -- cardinal B-spline shapes (section 2.2, the PIC shape function S)
  spectral  -- naive 2-D DFT, wavenumbers, spectral gradient / divergence
  steppers  -- BDF-k, CDF-2 and s-stage DIRK per-mode wave updates (section 3)
  pic       -- deposit, gather, IAEM push, initial state, Algorithm 1 step,
               residuals and energies (sections 2, 3, 4); 2D-2V or 2D-3V, one
               species or a species table
  adjoint   -- discrete adjoint of the step (BDF-k, the three CDF-2 forms, DIRK):
               gradients of the final magnetic energy (or final momenta) with respect
               to v^0 and P^0
  fixed_point -- bit-exact model of the FP32 form's move and fixed-point deposit

Every function is pinned by a ``-m "not gpu"`` test in ``tests/test_oracle_*.py``
against something the paper or plain mathematics fixes.
"""
