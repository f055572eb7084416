"""GB300-native Truncated Gaussian Basis Approach (arXiv:2410.04204).

The compute path is libtgba.so (CUDA for sm_103a, C ABI in include/tgba.h); ``tgba`` is its
thin Python binding.  Importing the package loads nothing; the first call into ``tgba``
loads the library and fails loudly if it has not been built.
"""
__all__ = ["tgba", "inputs", "build"]
