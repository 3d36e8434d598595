"""B300-native profile-likelihood library for trans-Gaussian geostatistical models.

The compute path lives in ``libplk.so`` (hand-written CUDA for sm_103a behind the
C ABI declared in ``include/plk.h``); ``paper_2305_04318_b300.native`` is the thin
ctypes binding.  ``synth`` generates seeded synthetic inputs.
"""
__all__ = ["native", "synth"]
