"""GB300-native block Lanczos with warm start (BLWS) for singular value thresholding.

The compute path is a C-ABI shared library of hand-written sm_103a CUDA kernels
(``csrc/``, declared in ``include/blws.h``); ``blws`` is its thin ctypes binding.
Importing this package loads nothing; the library is opened on first use.
"""
__all__ = ["blws", "synthetic"]
