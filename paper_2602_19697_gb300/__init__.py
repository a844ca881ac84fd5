"""GB300-native narrow-band posterior solver for probabilistic signed-distance
fusion (BayesFusion-SDF, arXiv 2602.19697).

The computation lives in the CUDA library ``libbfsdf.so`` (C ABI:
include/bfsdf.h); ``bfsdf`` is its Python binding.  Importing this package
loads nothing: call ``build.build()`` to compile and ``bfsdf.Context`` to use.
"""
__all__ = ["bfsdf", "build"]
