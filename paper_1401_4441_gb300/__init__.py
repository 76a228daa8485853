"""GB300-native link-cell Lennard-Jones force sweep with Newton's third law.

The compute path is the C-ABI library ``liblc.so`` (CUDA kernels for sm_103a,
declared in include/lc.h); ``paper_1401_4441_gb300.lc`` is its thin ctypes
binding.  Importing this package loads nothing; the library is loaded on the
first use of ``paper_1401_4441_gb300.lc``.
"""
