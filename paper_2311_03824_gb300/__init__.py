"""GB300-native AltGDmin-LR+S solver (arXiv 2311.03824): CUDA kernels for sm_103a
behind the C ABI of include/lrs.h, with a thin ctypes binding (lrs.py)."""
from .lrs import *  # noqa: F401,F403
from .lrs import Solver, LrsError, lib  # noqa: F401
