"""GB300 (sm_103a) reduced Wigner matrices and the fused beam-convolution l-sum.

The compute path is the CUDA library built from csrc/ (see build.py); this package
only marshals torch tensors to its C ABI (wigner.py) and wraps it for autograd.
"""
from .wigner import (  # noqa: F401
    WG_FP32X,
    WG_FP64,
    WignerError,
    check_device_status,
    load,
    wigner_conv_sum,
    wigner_conv_sum_backward,
    wigner_d_table,
    wigner_d_table_backward,
    wigner_device_status,
    wigner_fma_peak,
)
