"""GB300-native MHD + H/H2 chemistry time step (Kulikov, Chernykh & Protasov, arXiv:1608.08748).

The compute path is the CUDA library ``libmhd.so`` (C-ABI declared in ``include/mhd.h``); the
Python side (``mhd``) is argument marshalling only.  ``inputs`` builds seeded synthetic initial
states.
"""
from . import inputs  # noqa: F401
from .mhd import (Batch, MHDError, Server, Sim, bytes_needed, from_ic, lib, log_steps, probe_fma_peak,  # noqa: F401
                  profile)
