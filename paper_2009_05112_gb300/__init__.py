"""vegas+ (Lepage, arXiv:2009.05112) hot path on one GB300: a C-ABI CUDA library
(include/vegasp.h, ``libvegasp.so``) and its thin Python binding (``vegasp``).

``inputs`` holds the seeded synthetic workloads shaped like the paper's examples.
"""
__all__ = ["inputs", "vegasp", "build"]
