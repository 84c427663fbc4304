"""GB300-native (sm_103a) LLR density-of-states hot path for 4-D compact U(1).

The compute runs in the CUDA library built from ``csrc/`` and exposed through
the C ABI declared in ``include/llr.h``; ``llr.py`` is the thin ctypes
binding.  Importing this package does not load the library; ``llr.load()``
does, and fails loudly if it is missing.
"""
__all__ = ["llr", "workloads"]
