"""GB300-native (sm_103a) solver for the history integrals of the spherical mixed p-spin
dynamical mean-field equations on the non-uniform two-time grid (DYNAMITE, arXiv 2604.06309).

The computation lives in libdmfe.so (C ABI, include/dmfe.h); ``dmfe`` is its ctypes
binding and ``inputs`` holds the seeded synthetic input generators.
"""

from .dmfe import Batch, Server, Solver, DMFEError, fma_rate, footprint, load, theta_grid  # noqa: F401
