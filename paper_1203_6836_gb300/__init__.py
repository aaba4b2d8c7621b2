"""GB300-native Fast-QMMD / SP2 density-matrix hot path.

The computation lives in libtbmd.so (CUDA for sm_103a, C ABI in
include/tbmd.h); `tbmd` binds it with ctypes and `device` lays out torch
device memory for it.  `build.build()` compiles the library in-tree.
"""

__all__ = ["build", "tbmd", "device"]
