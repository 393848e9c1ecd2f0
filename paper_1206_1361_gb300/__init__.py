"""GB300 (sm_103a) split-step Crank-Nicolson solver for the time-dependent
Gross-Pitaevskii equation in an anisotropic harmonic trap.

The compute path is libgp.so (CUDA, C ABI in include/gp.h); ``gp`` is its
ctypes binding.  Importing this package does not load the library; the first
call does, and fails loudly if it has not been built.
"""
from . import gp  # noqa: F401
from .gp import (GP_C64, GP_C128, GP_IMAG, GP_REAL, GPError, Solver,  # noqa: F401
                 load_library)
