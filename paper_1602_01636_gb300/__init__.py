"""igafd: GB300-native PCG with a fast-diagonalization preconditioner for
single-patch isogeometric Poisson problems (Sangalli & Tani).

The compute path is the CUDA library ``libigafd.so`` (C ABI declared in
``include/igafd.h``); ``paper_1602_01636_gb300.igafd`` is a thin ctypes
binding that marshals torch device tensors and streams into it. Importing
the package does not load the library; ``igafd.lib()`` does, and raises if
the library has not been built.
"""
