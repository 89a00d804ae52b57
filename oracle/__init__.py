"""TEST INFRASTRUCTURE ONLY: the FP64 CPU oracle of the staggered RHMC.

Plain C (``stag_oracle.c``) loaded through ctypes, plus the Remez exchange in
``remez.py``.  Only the test suite, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package.  It shares no code with
the CUDA library in ``paper_1106_5673_gb300``.
"""
from .core import *  # noqa: F401,F403
