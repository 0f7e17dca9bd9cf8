"""GB300-native matrix-free pressure / viscous CG and time step of the
spectral semi-implicit staggered DG scheme (Fambri & Dumbser, Sec. 2).

The compute path is libsdg.so (hand-written CUDA for sm_103a behind the C ABI
of include/sdg.h); `sdg` is its ctypes binding.  Importing the package does
not load the library; the first call does, and fails loudly if it is missing.
"""
from . import sdg  # noqa: F401

__all__ = ["sdg"]
