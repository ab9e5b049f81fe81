"""GB300-native inverse-free SVGP (R-SVGP) training step.

The compute path is ``libsvgp.so`` (hand-written CUDA for sm_103a) behind the
C-ABI in include/svgp.h; ``_lib`` is its ctypes binding and ``model`` a thin
device-state helper.  Importing this package does not load the library.
"""
__all__ = ["build", "_lib", "model"]
