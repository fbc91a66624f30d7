"""CPU oracle for RbmSAT (test infrastructure only; see rbmsat.py)."""
from .rbmsat import *  # noqa: F401,F403
from .rbmsat import build, lib  # noqa: F401
