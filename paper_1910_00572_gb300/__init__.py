"""GB300 belief-tensor localizer (map-corrected odometry, arXiv 1910.00572).

The compute path is the CUDA library ``libloc.so`` built from ``csrc/`` for sm_103a; this
package is a thin ctypes binding over its C-ABI (``include/loc.h``) with the same names.
There is no CPU fallback: every function raises if the library is missing.
"""
from .binding import *  # noqa: F401,F403
from .binding import __all__  # noqa: F401
