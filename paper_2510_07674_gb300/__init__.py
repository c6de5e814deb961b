"""GB300-native SPaSM hot path: CUDA kernels behind a C ABI, with a thin ctypes binding.

Importing the package loads nothing; ``paper_2510_07674_gb300.spasm`` loads the CUDA
library and fails loudly if it was not built.
"""
__all__ = ["scenes"]
