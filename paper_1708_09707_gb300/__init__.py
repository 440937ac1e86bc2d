"""GB300-native H-matrix build and H-matrix-vector product for kernel matrices.

The compute path lives in the CUDA shared library ``libhm.so`` (sources under
``csrc/``, C-ABI declared in ``include/hm.h``); ``paper_1708_09707_gb300.hm``
is the thin ctypes binding over it. Importing this package loads nothing.
"""
