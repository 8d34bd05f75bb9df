"""GB300-native counter-guided tuning-space search step (arXiv 2102.05297).

The compute path lives in libktune.so (CUDA, sm_103a) behind the C ABI of
include/ktune.h; ``paper_2102_05297_gb300.ktune`` is its ctypes binding and
``paper_2102_05297_gb300.fit`` the host-side model tooling.  Importing the
binding fails loudly if the library is not built.
"""
__all__ = ["ktune"]
