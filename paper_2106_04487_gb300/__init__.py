"""GB300-native Fast Kernel Transform (arXiv 2106.04487): y = Ktilde(X, X) w on a spatial tree.

The compute path is the C-ABI library ``libfkt.so`` (hand-written sm_103a CUDA,
declared in ``include/fkt.h``); ``fkt`` is its thin ctypes binding.  Importing
this package does not load the library; ``fkt.lib()`` does, and raises if it
is missing -- there is no CPU fallback.
"""
__all__ = ["fkt", "inputs"]
