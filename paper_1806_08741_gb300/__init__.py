"""GB300-native Scalable SLIC (SSLIC) superpixels / supervoxels.

The method (arXiv 1806.08741) runs as hand-written CUDA kernels for sm_103a
behind the C ABI declared in ``include/sslic.h``; ``sslic`` is the thin
ctypes binding to that library.
"""
