"""sp-DBA oracle: a plain, slow, FP64 CPU implementation of the method.

TEST INFRASTRUCTURE.  Only tests/, the smoke check in __graft_entry__ and the
CPU-baseline / reference legs of bench.py may import this package.  It shares
no code with the CUDA path and imports nothing from it.
"""
from .spdba_oracle import *  # noqa: F401,F403
