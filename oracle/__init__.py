"""Plain, slow, FP64 CPU oracle for Generative Monte Carlo.

TEST INFRASTRUCTURE ONLY. Only the tests, `__graft_entry__.smoke()` and the
CPU-baseline leg of `bench.py` may import or run anything in this package.
It shares no code with the CUDA path and imports nothing from it.

Modules (each cites the passage of the paper it follows):
  rng        Philox4x32-10 (Salmon et al., SC'11), uniforms in (0,1] (Eq. 4),
             Box-Muller normals (the Gaussian seeds of Eq. 8).
  transport  random-walk cell transmission (Eq. 4-6, analog and implicit
             capture), standard MC solve (Eq. 5-7), event-based GMC solve (the
             four stages of the transport algorithm).
  mlp        velocity network, fixed-step flow ODE (Eq. 8), exit-state
             decoding (Eq. 10-11).
  train      CFM loss (Eq. 9), its gradient, AdamW.
  stats      moments, 1-D Wasserstein distance, Eq. 12.

Parity pins: every function is pinned by a CPU test against closed forms,
published values, invariants or library routines (see tests/test_oracle_*.py).
"""
from . import rng, transport, mlp, train, stats  # noqa: F401
from ._clib import build  # noqa: F401
