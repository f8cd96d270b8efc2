"""GB300-native max-pooling path planner (arXiv 2004.00540, oMAP).

The CUDA library libmpn.so (C ABI in include/mpn.h) does all the work:
bit-packed encoding of the environment map, the stack of max-pool layers as a
temporally blocked persistent bit-plane wavefront, and warp-per-start path
reconstruction. ``mpn`` is its thin ctypes binding.
"""
from .mpn import *  # noqa: F401,F403
from .mpn import Planner, Paths, MPNError, load, EXPORTS  # noqa: F401
