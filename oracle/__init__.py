"""FP64 CPU oracle for field-dependent coronagraphic image simulation.

TEST INFRASTRUCTURE ONLY.  Plain, slow, obviously correct NumPy written from
the paper (Sec. 2: interpolated PSF library; Sec. 3: S = A Z).  It shares no
code with the CUDA path and neither imports the other.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference leg may
import it; the product path must never route through it.

Modules:
  psfsim_oracle  geometry (Eq. 2-3), radial lerp, bilinear rotation, A, A x, A^T g
  ring_oracle    exozodi ring model, its analytic parameter gradient, the fit loss
  split_oracle   split-BF16 (hi + lo with per-column power-of-two scale) encoding
  convolution_oracle  direct FP64 convolution (the Sec. 3 comparison system)

Parity status: every function is pinned by ``tests/test_oracle_*.py`` against
closed forms, invariants, brute force or library routines (see each docstring).
"""
