"""GB300 (sm_103a) RbmSAT: block Gibbs sampling of a formula RBM for MaxSAT
("Solving MaxSAT with Matrix Multiplication"), behind the C ABI of
include/maxsat.h. This package holds the CUDA/C++ sources (csrc/), the build
step (build.py) and the ctypes binding (binding.py)."""
from .binding import *  # noqa: F401,F403
from .binding import Context, MaxsatError, lib  # noqa: F401
