"""GB300-native even-odd twisted-mass clover operators and Krylov solvers.

The compute lives in libtm.so (C ABI declared in include/tm.h, CUDA kernels
for sm_103a in csrc/); ``paper_2212_06635_gb300.tm`` is its ctypes binding.
"""
