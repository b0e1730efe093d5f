"""FP64 CPU oracle of one cRKFR step (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py``
may import this package.  It shares no code with the CUDA library.
"""
from .oracle import *  # noqa: F401,F403
