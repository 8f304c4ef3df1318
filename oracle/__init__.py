"""FP64 CPU oracle: test infrastructure, not part of the library.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path.
"""
from .dfb_oracle import *  # noqa: F401,F403
