"""GB300 implementation of history-free collision response (J. Ye,
arXiv 1409.2081): exact edge-face discrete collision detection, penetration
stencils and the global displacement minimizer, behind the C ABI declared
in include/hfcr.h.  `api` is the ctypes binding; `build` compiles the
library for sm_103a."""
from . import api  # noqa: F401
