"""GB300-native hot path of two-flavour staggered RHMC (arXiv:1106.5673).

The compute path is libstag.so (hand-written sm_103a CUDA behind a C ABI,
include/stag.h); ``stag`` is its thin ctypes binding.  There is no CPU
fallback: importing ``stag`` raises if the library is missing.
"""
from . import synth  # noqa: F401
