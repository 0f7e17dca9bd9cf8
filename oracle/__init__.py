"""CPU FP64 oracle of the staggered DG pressure/viscous/step path.

Test infrastructure: only tests, the smoke check and the benchmark's CPU
baseline leg use it.  It shares no code with the CUDA library.
"""
from .sdg_oracle import *  # noqa: F401,F403
from .sdg_adjoint import Adjoint  # noqa: F401
