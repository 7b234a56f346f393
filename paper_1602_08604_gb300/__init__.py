"""GB300-native LRE hot path for full quantum state tomography (arXiv:1602.08604).

The compute lives in liblre.so (CUDA C++ for sm_103a) behind the C ABI in
include/lre.h; `paper_1602_08604_gb300.lre` is a thin ctypes binding with
the same names.  There is no CPU fallback: importing the binding without
the built library raises.
"""
