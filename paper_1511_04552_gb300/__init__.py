"""GB300-native (sm_103a) MCLBM: one time step of the twin-component lattice Boltzmann model
of buoyancy-driven convection in a nanosuspension (arXiv:1511.04552), as a CUDA library with
a C ABI (include/mclbm.h) and this thin Python binding."""
from .binding import (  # noqa: F401
    Batch, Cavity, MclbmError, sweep_to_steady, Props, create, get_consts, lib, props_default, run_to_steady,
    steady_nu_reached,
    F_ALL, F_BROWNIAN, F_BUOYANCY, F_DRAG, F_GRAVITY, F_MAGNUS, F_SAFFMAN, F_THERMOPHORESIS,
    UX, UY, THETA, PHI, RHO_W, RHO_P, UPX, UPY, INIT_REST, INIT_WARM, INIT_WARM_RHO, EXPORTS,
    STORE_F32, STORE_F16, STORE_BF16, ROUND_STOCHASTIC, ROUND_NEAREST,
)
