"""GB300 (sm_103a) XPCS two-time correlation on raw and homomorphically compressed frames.

The compute lives in ``lib/libxpcs.so`` (C ABI in ``include/xpcs.h``); ``xpcs`` is its
ctypes binding.  Importing ``paper_2407_20356_gb300.xpcs`` fails loudly if the library
has not been built.
"""
__all__ = ["xpcs"]
