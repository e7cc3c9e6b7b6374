"""GB300-native dSASA: exact inclusion-exclusion SASA and its gradient on one GPU.

The compute path lives in the CUDA library ``_build/libdsasa.so`` (sources in ``csrc/``,
C ABI in ``include/dsasa.h``); ``api`` is the thin ctypes binding over it.
Importing this package does not load CUDA; ``api`` does, and fails loudly if the
library is missing.
"""
__all__ = ["inputs"]
