"""CPU oracle for the Lie-closure hot path (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  It shares no code with the CUDA library.
"""
from .closure import *  # noqa: F401,F403
