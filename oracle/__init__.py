"""FP64 CPU oracle of the twin-component lattice Boltzmann model (MCLBM) step.

TEST INFRASTRUCTURE. Only tests/, the smoke check and bench.py's CPU-baseline leg may import
this package. The product path (the CUDA library and its binding) never imports it and shares
no code with it.
"""
from .ref import *  # noqa: F401,F403
from .ref import RefSolver, RefError, default_props, equilibrium, drag_impulse  # noqa: F401
from .build import build  # noqa: F401
