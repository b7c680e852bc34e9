"""FP64 CPU oracle of AltGDmin-LR+S (arXiv 2311.03824, Algorithms 1 and 2).

TEST INFRASTRUCTURE: imported only by the tests, the smoke check and the
benchmark's CPU-baseline leg.  The solver library never uses it.
"""
from .altgdmin_lrs import *  # noqa: F401,F403
