"""psfsim: GB300-native field-dependent coronagraphic image simulation.

The interpolated-PSF-library method of Milani & Douglas (Sec. 2-3): a radial
library of off-axis PSFs is interpolated in offset and rotated to every scene
pixel, giving A whose column j is pixel j's PSF; an image is S = A Z.

Layout:
  csrc/        CUDA kernels (sm_103a) and the C ABI of libpsfsim.so
  _binding.py  ctypes declarations of include/psfsim*.h
  plan.py      Plan: build / forward / adjoint on torch-owned device memory
  build_lib.py compiles csrc/ in-tree
"""
from ._binding import PsfsimError, load  # noqa: F401
from .plan import Plan, workspace_bytes  # noqa: F401
