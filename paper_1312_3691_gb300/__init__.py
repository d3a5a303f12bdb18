"""GB300-native TPMC hot path (Parham & Barba, arXiv 1312.3691).

The compute path lives in libtpmc.so (hand-written CUDA for sm_103a plus a C++
host runtime) behind the C ABI of include/tpmc.h; ``tpmc`` is its ctypes
binding with the same function names.  Build with ``paper_1312_3691_gb300.build.build()``.
"""
from . import tpmc  # noqa: F401

