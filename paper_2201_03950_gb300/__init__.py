"""GB300-native (sm_103a) batched tridiagonal solver and ADI heat-diffusion step.

The compute path is hand-written CUDA behind a C ABI (``include/trid.h``); the
Python layer in ``trid`` only marshals pointers, sizes and the CUDA stream.
"""
