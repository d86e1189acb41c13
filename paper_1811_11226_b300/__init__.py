"""B300-native CT data augmentation (arXiv 1811.11226, Sec. 4 and 5.C).

The compute path is the CUDA library ``libaugwarp.so`` (C ABI in
``include/augwarp.h``); :mod:`.augwarp` is its Python binding.  Importing the
binding fails loudly when the library has not been built.
"""

__all__ = ["augwarp", "build"]
