"""FP64 CPU oracle of the two-fluid lattice step (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may import
this package.  It shares no code with the CUDA library.
"""
from . import twofluid  # noqa: F401
