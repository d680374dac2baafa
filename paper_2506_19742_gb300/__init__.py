"""GB300-native NeRF-CBCT training step ("NeRF-based CBCT Reconstruction needs
Normalization and Initialization"): hand-written CUDA kernels for sm_103a behind
the C ABI in include/nhcbct.h, with a thin ctypes binding in ``nhcbct``.

Importing the package loads nothing; ``nhcbct.load()`` (called by every entry
point) loads the built library and raises if it is missing.
"""
__all__ = ["nhcbct", "build"]
