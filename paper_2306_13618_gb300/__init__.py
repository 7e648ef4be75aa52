"""GB300-native radial Gaussian kernel summation for entropic unbalanced
optimal transport and MMD (arXiv 2306.13618).

The compute path is the CUDA C-ABI library ``_lib/libuotk.so`` (sources in
``csrc/``, declarations in ``include/uotk.h``); ``uotk`` is its thin ctypes
binding.  Importing this package does not load the library: ``uotk.lib()``
does, and raises if it has not been built.
"""
__all__ = ["uotk", "inputs"]
