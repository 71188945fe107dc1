"""GB300-native proton Monte Carlo dose engine.

Implements the condensed-history proton transport method of Wan Chan Tseung,
Ma & Beltran (arXiv:1409.8336) as hand-written sm_103a CUDA kernels behind a
C ABI (include/pmc.h).  `Engine` is the thin Python binding of that ABI;
`workloads` holds the seeded synthetic inputs.
"""
from .engine import (FULL_CASCADE, NO_ELASTIC, NO_INELASTIC, NO_MCS, NO_STRAGGLING, SURROGATE, Engine, GammaIndex,
                     PlanStream, PmcError, debug_philox, gamma_index)

__all__ = ["Engine", "PlanStream", "PmcError", "GammaIndex", "gamma_index", "debug_philox", "FULL_CASCADE", "SURROGATE", "NO_STRAGGLING", "NO_MCS",
           "NO_ELASTIC", "NO_INELASTIC"]
