"""GB300-native two-fluid active-nematic / passive-fluid lattice solver.

The computation lives in the CUDA library libtwofluid.so (C ABI in
include/twofluid.h); this package holds its build script, a thin ctypes
binding and the seeded synthetic-input generators.  Importing the package
does not load the library; ``TwoFluid`` does, and raises if it is missing.
"""
from ._binding import (  # noqa: F401
    EXPORTS, FIELD_F1, FIELD_F2, FIELD_MU, FIELD_PHI, FIELD_QXX, FIELD_QXY, FIELD_RHO1,
    FIELD_RHO2, FIELD_U1X, FIELD_U1Y, FIELD_U2X, FIELD_U2Y, NCONS, SolverParams, TwoFluid,
    TwoFluidError, load_library,
)
