"""BinSketch on GB300: CUDA kernels behind a C ABI, with a thin Python binding.

Importing the package does not load the CUDA library; ``binding.lib()`` does,
and raises if it has not been built (no CPU fallback exists).
"""
__version__ = "0.1.0"
