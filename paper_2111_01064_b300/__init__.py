"""B300-native batched LISA likelihood for massive-black-hole-binary templates
(arXiv:2111.01064, Sec. II): CUDA kernels for sm_103a behind the C ABI of
include/mbhlike.h, and a thin ctypes binding (``mbhlike``) with the same names.

Importing the package loads nothing; the first call into ``mbhlike`` loads
libmbhlike.so and raises if it is missing or no CUDA device is usable.
"""
__all__ = ["mbhlike"]
