"""GB300-native unsplit geometric VOF hot path (LSGIR + FMFPA).

The compute path is the CUDA library ``libgvof.so`` (C-ABI, declared in
``include/vof.h``); ``paper_2111_01524_gb300.vof`` is its thin ctypes
binding. Importing this package loads nothing: the library is opened on first
use and the binding raises if it is missing.
"""
__all__ = ["inputs", "vof"]
