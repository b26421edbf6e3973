"""GB300-native error-bounded multilevel (MGARD-style) compressor.

The compute path lives in ``libhpdr.so`` (hand-written sm_103a CUDA behind a
C ABI declared in ``include/hpdr.h``); ``hpdr`` is its thin Python binding.
Importing this package does not load the library; the first call does, and
fails loudly if it is missing.
"""
__all__ = ["hpdr", "fields"]
