"""GB300-native exact filtered vector search (arXiv 2403.15807 scan path).

The search runs in libvrs.so (CUDA kernels for sm_103a behind the C ABI of
include/vrs.h); ``paper_2403_15807_gb300.vrs`` is the ctypes binding and
``paper_2403_15807_gb300.build`` compiles the library in-tree.
"""
__all__ = ["vrs", "build"]
