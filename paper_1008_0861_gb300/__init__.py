"""GB300 (sm_103a) implementation of the directionally split semi-implicit
anisotropic-diffusion step (Sharma & Hammett, arXiv:1008.0861, Section 2).

The method runs in libaniso.so (hand-written CUDA kernels behind the C ABI of
include/aniso.h); this package is its thin Python binding, with the same
function names as the C ABI.  PyTorch is only used by callers for device
memory and streams."""
from ._binding import *  # noqa: F401,F403
from ._binding import load, AnisoError, LIB_PATH, EXPORTED  # noqa: F401
