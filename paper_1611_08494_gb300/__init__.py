"""GB300-native sky cross-match (paper arXiv:1611.08494, §2.1 Sky functional
case, §2.2 match selection and joins, §2.3 sky partitioning).

The compute path is the CUDA library ``_lib/libxm.so`` (C ABI declared in
``include/xm.h``); ``xm`` is its thin ctypes binding. Importing the package
does not load the library; ``paper_1611_08494_gb300.xm`` does, and fails
loudly when it is missing.
"""
