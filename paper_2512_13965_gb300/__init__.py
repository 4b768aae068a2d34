"""GB300-native Generative Monte Carlo: Python binding of libgmc.so.

The compute path is the CUDA library (include/gmc.h); this package only
loads it and marshals arguments. Importing it without the built library
raises ImportError.
"""
from ._abi import *  # noqa: F401,F403
from ._abi import (Context, GMCError, gmc_config, gmc_solve_stats, lib,  # noqa: F401
                   LIB_PATH)
